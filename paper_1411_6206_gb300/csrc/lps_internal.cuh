// Internal declarations shared by the kernels and the host side of liblps.so.
// Device helpers: complex arithmetic, bounded mbarrier waits, 1D TMA bulk copies,
// shared-memory Stockham FFT passes and deterministic block reductions.
#pragma once

#include <cstdint>
#include <utility>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace lps {

constexpr int kThreads = 256;          // threads per CTA of the per-plane and per-tile kernels
constexpr int kMaxPasses = 8;          // radix passes per transform length
constexpr int kTile = 8;               // in-plane tile edge of the sparse-step kernel
constexpr int kMaxNc = 32;             // largest Casorati column count
constexpr long long kSpinLimit = 1LL << 26;   // bounded waits: iterations before giving up

// Status bits written by kernels into DevCtrl::err.
constexpr int kErrTimeout = 1;
constexpr int kErrNonfinite = 2;

struct FftPlan {
  int n;
  int np;                   // number of passes
  int r[kMaxPasses];        // radix of each pass, first to last
};

// Per-plan values that persist across frames (written by the host API).
struct DevPersist {
  int nlines;               // sampled lines of the current mask
  int has_sup;              // prior support present (nonzero)
  int has_sigma;            // prior singular values present (nonzero)
  int skip;                 // nonzero: the next frame is skipped (inactive member of a batch)
  int v_valid;              // eigenvectors from an earlier eigendecomposition are available
};

// Per-frame control block (zeroed at the start of every frame).
struct DevCtrl {
  float lambda_L, lambda_S;
  unsigned haar_max_bits;   // max |T(X_0)| as float bits (non-negative, order-preserving)
  int lambdas_set;
  int converged;
  int iters_done;
  int err;
  int rank_cur;
  int sweeps_cur;           // Jacobi sweeps of the current eigendecomposition
  double sigma_max;
  double nuclear_cur;
};

// Per-iteration record as the eigen kernel writes it (no float64 arithmetic on the device:
// the host widens the float32 fields and forms the objective from them and the lambdas).
struct IterRec {
  double nuclear;
  float resid2, l1, rel_change;
  int rank, sweeps;
};

// objective of Sec. 3: ||E(L+S) - d||^2 / 2 + lambda_L ||L||_* + lambda_S ||T S||_1 (off the prior support)
inline double iter_objective(const IterRec& r, float lambda_L, float lambda_S) {
  return 0.5 * (double)r.resid2 + (double)lambda_L * r.nuclear + (double)lambda_S * (double)r.l1;
}

struct Geom {
  int nx, ny, nz, ncoil;    // nx: the x-planes this plan holds (a slab of nxt planes)
  int nxt, x0;              // x extent of the whole volume (readout length) and the slab's first plane
  int nc;                   // Casorati columns (nz / cs)
  int plane;                // ny*nz, elements of one x-plane
  int nyp;                  // padded row stride of the FFT buffers (odd)
  int planeP;               // nz*nyp rounded up to even
  int mpad;                 // row stride (elements) of the hybrid data per (x, coil)
  int fft_z;                // 3D (1) or per-slice 2D (0) encode
  int cs;                   // slices per Casorati column (> 1: columns are 3D frame volumes)
  int zn;                   // length of each z transform (nz, or cs for 3D frames)
  int J;                    // Haar levels
  int wz;                   // 1: 3D Haar (the 2D pyramid times the 1D Haar along z), 0: per slice
  int ntiles;               // (nx/8)*(ny/8)
  long long N;              // nx*ny*nz
  float scale_yz;           // 1/sqrt(ny*nz) (fft_z) or 1/sqrt(ny)
  float scale_x;            // 1/sqrt(nxt)
  FftPlan py, pz, px;
  int dc_generic;           // 1: always the runtime-sized data-consistency kernel (autotuner)
  int dc_direct;            // runtime-sized kernel reads coil maps from global memory (no staging)
  int lrs_tpc;              // 8x8 tiles per CTA of the sparse-step kernel (0: 32 / nc)
  int dc_reg_groups;        // register-transform DC kernel (128 x 16 planes): coil groups, 0 = off
  int dc_rt;                // update on k_dc's register-transform coil loop where the plane has one
  int dc_rt_dsm;            // that loop's shared-memory slots for a coil's samples (set at launch)
};

// ---- data-consistency / adjoint / forward kernel (one CTA per x-plane) -------------
enum DcMode { kDcUpdate = 0, kDcAdjoint = 1, kDcForward = 2 };

struct DcArgs {
  Geom g;
  const float2* L;          // update (operator form): Z = L + S;  forward: image
  const float2* S;          // update: S (the iteration's new sparse part; Gram of X - S)
  // Iteration form of the update (Algorithm 1): L_k is formed here, Z = L_k + S_k, and
  // X_{k-1} is read from X before X_k is written there.
  const float2* W;          // [nc][nc]: L_k = (X_{k-1} - S_{k-1}) W in the prologue
  const float2* Lpre;       // or L_k precomputed (tensor-core reprojection)
  const float2* Sprev;      // S_{k-1}
  float2* Lbuf;             // in: L_{k-1} (change statistic), out: L_k
  float2* X;                // update/adjoint: output X
  float2* L_out;            // adjoint: also write X_0 here (L_0 := X_0)
  float2* S_out;            // adjoint: zero S
  float2* recon;            // update: optional copy of Z = L + S
  const float2* coils;      // [ncoil][nz][nx][ny]
  const __half2* coils_h;   // the same maps in half precision (LPS_COILS_FP16), else nullptr
  const __half2* dhyb_h;    // the hybrid samples in half precision (LPS_DATA_FP16), else nullptr
  int* err_word;            // error flags when ctrl is null (operator calls), else nullptr
  int stall_polls;          // test hook (staged-coil kernel): > 0 makes the first coil wait on an
                            // mbarrier that nothing completes, with this poll budget
  const float2* dhyb;       // [nx][ncoil][mpad] hybrid-space samples
  float2* hyb_out;          // forward: [nx][ncoil][mpad]
  const int* lines;         // padded in-plane position kz*nyp + ky of each line
  const float2* tw_y;
  const float2* tw_z;
  float2* gram_part;        // [nx][nc][nc]; nullptr = skip
  float* dc_part;           // [nx][4]: ||E Z - d||^2, ||Z_k - Z_{k-1}||^2, ||Z_{k-1}||^2, 0; nullptr = skip
  const DevPersist* persist;
  DevCtrl* ctrl;            // nullptr = no convergence gating
};

// ---- hybrid transform along x --------------------------------------------------------
struct XfftArgs {
  Geom g;
  const float2* in;
  float2* out;
  const float2* tw_x;
  const DevPersist* persist;
  int inverse;              // 1: k-space [c][l][kx] -> hybrid [x][c][l] (the plan's planes x0 .. x0+nx-1);
                            // 0: the reverse (planes outside the slab count as zero)
};

// ---- support-aware sparse step (step 3), one CTA per group of 8x8 tiles ------------
struct LrsArgs {
  Geom g;
  const float2* X;          // X_{k-1}
  const float2* L;          // L_{k-1}
  float2* S;                // out: S_k
  const uint32_t* sup_prior;
  uint32_t* sup_out;        // nullptr = do not write the support bitmap
  float* lrs_part;          // [CTAs][2]: l1 off the prior support, support count
  const DevPersist* persist;
  DevCtrl* ctrl;
  double lambda_S_rel;      // lambda_S = lambda_S_rel * max |T(X_0)| until the lambdas are set
  int support_rule;
  int haar_max_only;        // 1: only max |T(X)| into ctrl->haar_max_bits
};

// ---- Gram reduction + eigendecomposition + SVT + prior pull (one CTA) --------------
struct EigArgs {
  Geom g;
  const float2* gram_part;  // [nparts][nc][nc]
  int nparts;
  const float* dc_part;     // [ndc][4]
  int ndc;                  // data-consistency statistic partials (nx; 1 for a reduced slab record)
  const float* lrs_part;    // [lrs_parts][2]
  int lrs_parts;            // CTAs of the sparse-step kernel
  float2* W;                // [nc][nc]
  float2* V;                // [nc][nc] warm-start eigenvectors
  const double* sigma_prev;
  double* sigma_out;        // sigma'' in rank order
  IterRec* hist;
  DevPersist* persist;      // v_valid is set once eigenvectors exist
  DevCtrl* ctrl;
  double lambda_L_rel, lambda_S_rel, lambda_p, rank_tau, tol;
  float lambda_p_f, rank_tau_f, tol_f;   // the same three rounded to float32 (float32 path)
  int iter;                 // iteration k whose SVT this launch computes (1-based)
  int finalize;             // 1: only record the stats of iteration `iter`-1
  int eig_fp64;
  // float64 mode: part 1 (statistics, Gram, float32 Jacobi) hands off to the float64
  // Rayleigh-Ritz kernels, part 2 (singular-value steps and W) continues from their output
  int part;                 // 0: whole kernel; 1 or 2
  float2* Gout;             // part 1: the Gram [nc][nc]
  double* lam64;            // part 1 out: float32 eigenvalues; part 2 in: float64 ones
  const float2* Vin;        // part 2: refined eigenvectors (else the warm start is V)
};

// ---- float64 Rayleigh-Ritz refinement of the float32 eigendecomposition ------------
struct RitzArgs {
  int n;
  const float2* G;          // [n][n]
  const float2* V;          // [n][n] float32 eigenvectors (columns)
  double2* A;               // [n][n] A = V^H G V (float64)
  float2* Vout;             // [n][n] refined eigenvectors
  double* lam64;            // [n] refined eigenvalues
  const DevCtrl* ctrl;
};
cudaError_t launch_ritz64(const RitzArgs& a, cudaStream_t st);

// ---- tensor-core contractions of the precision modes (tcgen05) ----------------------
constexpr int kPrecTf32 = 1;   // = LPS_TF32_REFINE
constexpr int kPrecBf16 = 2;   // = LPS_BF16_REFINE
struct GramTcArgs {
  Geom g;
  const float2* X;
  const float2* S;          // nullptr: S = 0
  float2* gram_part;        // [gram_tc_parts][nc][nc]
  DevCtrl* ctrl;
};
struct ReprojTcArgs {
  Geom g;
  const float2* X;
  const float2* S;
  const float2* W;          // [nc][nc]
  float2* Lnew;             // (X - S) W
  DevCtrl* ctrl;
};

// Host-side launchers (return cudaGetLastError()).
cudaError_t launch_dc(const DcArgs& a, int mode, cudaStream_t st);
cudaError_t launch_xfft(const XfftArgs& a, cudaStream_t st);
cudaError_t launch_lrs(const LrsArgs& a, cudaStream_t st);
cudaError_t launch_eig(const EigArgs& a, cudaStream_t st);
size_t dc_smem_bytes(const Geom& g);
size_t xfft_smem_bytes(const Geom& g);
int dc_ept(const Geom& g);
int lrs_blocks(const Geom& g);
int lrs_tpc(const Geom& g);
int lrs_threads(const Geom& g);
bool dc_has_fixed(const Geom& g);
bool dc_reg_applies(const Geom& g);
bool dc_rt_geometry(const Geom& g);   // a register-transform instantiation exists for the plane
bool dc_rt_applies(const Geom& g);
// persistent batch form of the update (operator form): one launch over a descriptor table
bool dc_persist_fits(const Geom& g);
size_t dc_persist_smem(const Geom& g);
cudaError_t launch_dc_persist(const DcArgs* table, const int* start, int nm, int* counter, size_t smem,
                              cudaStream_t st);
cudaError_t launch_dc_reg(const DcArgs& a, cudaStream_t st);
int dc_gram_parts(const Geom& g);
int gram_tc_parts(const Geom& g);
cudaError_t launch_gram_sum(const float2* part, int nparts, int nc, float2* G, cudaStream_t st);
// Rounds n complex values to half precision: h = the rounded pairs, c rewritten with their
// float32 values (so that every kernel reads the same maps).
cudaError_t launch_round_half(float2* c, __half2* h, long long n, cudaStream_t st);
cudaError_t launch_settle(const DevCtrl* ctrl, int k0, float2* S0, const float2* S1, long long n, uint32_t* sup0,
                          const uint32_t* sup1, long long nw, float* part0, const float* part1, int np,
                          cudaStream_t st);
cudaError_t launch_reproj_f32(const float2* X, const float2* S, const float2* W, float2* L, const Geom& g,
                              cudaStream_t st);
cudaError_t launch_gram_tc(const GramTcArgs& a, int precision, cudaStream_t st);
cudaError_t launch_reproj_tc(const ReprojTcArgs& a, int precision, cudaStream_t st);

// Launch with programmatic stream serialization: the kernel may start while its predecessor
// in the stream finishes; it must call pdl_wait() before reading the predecessor's outputs.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace lps

#ifdef __CUDACC__
namespace lps {

// Programmatic dependent launch: wait for the predecessor grid (and its memory) / allow the
// successor grid to be scheduled. Both are no-ops without the launch attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---- complex helpers ---------------------------------------------------------------
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// multiply by -i (forward) or +i (inverse)
__device__ __forceinline__ float2 mul_mi(float2 a, bool inv) {
  return inv ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// ---- shared-memory addresses, mbarriers and 1D bulk copies (TMA) ----------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: returns false (and records kErrTimeout) if the phase never completes within
// `limit` polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, int* err,
                                                  long long limit = kSpinLimit) {
  for (long long i = 0; i < limit; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (i > 64) __nanosleep(64);
  }
  if (err) atomicOr(err, kErrTimeout);
  return false;
}

// ---- deterministic reductions -------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}
// Sum over the block in a fixed order; result valid in thread 0. `red` holds >= 32 floats.
__device__ __forceinline__ float block_sum(float v, float* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  float r = 0.f;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) r += red[i];
  }
  return r;
}
__device__ __forceinline__ float block_max(float v, float* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  float r = 0.f;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) r = fmaxf(r, red[i]);
  }
  return r;
}

// ---- small DFTs in registers (forward: exp(-2 pi i rs/R), inverse: +) -----------------
__device__ __forceinline__ void dft2(float2& a, float2& b) {
  float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}
__device__ __forceinline__ void dft4(float2* v, bool inv) {
  float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
  float2 t2 = cadd(v[1], v[3]), t3 = mul_mi(csub(v[1], v[3]), inv);
  v[0] = cadd(t0, t2);
  v[2] = csub(t0, t2);
  v[1] = cadd(t1, t3);
  v[3] = csub(t1, t3);
}
// v[0..7]: two radix-4 DFTs on even/odd samples and one radix-2 stage.
__device__ __forceinline__ void dft8(float2* v, bool inv) {
  const float h = 0.70710678118654752f;   // sqrt(2)/2
  float2 e[4] = {v[0], v[2], v[4], v[6]};
  float2 o[4] = {v[1], v[3], v[5], v[7]};
  dft4(e, inv);
  dft4(o, inv);
  // twiddles w8^k, k = 0..3: 1, h(1 -+ i), -+i, h(-1 -+ i)
  float2 o1 = inv ? make_float2(h * (o[1].x - o[1].y), h * (o[1].x + o[1].y))
                  : make_float2(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x));
  float2 o2 = mul_mi(o[2], inv);
  float2 o3 = inv ? make_float2(-h * (o[3].x + o[3].y), h * (o[3].x - o[3].y))
                  : make_float2(h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y));
  v[0] = cadd(e[0], o[0]);
  v[4] = csub(e[0], o[0]);
  v[1] = cadd(e[1], o1);
  v[5] = csub(e[1], o1);
  v[2] = cadd(e[2], o2);
  v[6] = csub(e[2], o2);
  v[3] = cadd(e[3], o3);
  v[7] = csub(e[3], o3);
}
// v[0..15]: two radix-8 DFTs on even/odd samples and one radix-2 stage with w16^k.
__device__ __forceinline__ void dft16(float2* v, bool inv) {
  float2 e[8], o[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    e[i] = v[2 * i];
    o[i] = v[2 * i + 1];
  }
  dft8(e, inv);
  dft8(o, inv);
  // cos(k pi/8), sin(k pi/8) for k = 0..7
  const float C[8] = {1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f,
                      0.0f, -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128674f};
  const float S[8] = {0.0f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128674f,
                      1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f};
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    float2 w = make_float2(C[k], inv ? S[k] : -S[k]);
    float2 t = cmul(o[k], w);
    v[k] = cadd(e[k], t);
    v[k + 8] = csub(e[k], t);
  }
}
// Generic radix-R DFT, roots taken from the length-n table (R divides n).
template <int R>
__device__ __forceinline__ void dft_generic(float2* v, bool inv, const float2* tw, int n) {
  float2 out[R];
  const int st = n / R;
#pragma unroll
  for (int s = 0; s < R; ++s) {
    float2 acc = v[0];
#pragma unroll
    for (int r = 1; r < R; ++r) {
      float2 w = tw[((r * s) % R) * st];
      if (inv) w.y = -w.y;
      acc = cadd(acc, cmul(v[r], w));
    }
    out[s] = acc;
  }
#pragma unroll
  for (int s = 0; s < R; ++s) v[s] = out[s];
}

template <int R>
__device__ __forceinline__ void dft_reg(float2* v, bool inv, const float2* tw, int n) {
  if constexpr (R == 2) {
    dft2(v[0], v[1]);
  } else if constexpr (R == 4) {
    dft4(v, inv);
  } else if constexpr (R == 8) {
    dft8(v, inv);
  } else if constexpr (R == 16) {
    dft16(v, inv);
  } else {
    dft_generic<R>(v, inv, tw, n);
  }
}

// Division by a divisor fixed for a whole pass: q = floor(t * m / 2^32) with m = ceil(2^32 / d)
// is floor(t / d) or one more (for t < 2^32), corrected once.
struct FastDiv {
  unsigned d, m;
};
__device__ __forceinline__ FastDiv make_fdiv(unsigned d) {
  return FastDiv{d, d > 1 ? (unsigned)(0xFFFFFFFFull / d + 1ull) : 0u};
}
__device__ __forceinline__ unsigned fdiv(unsigned t, FastDiv f) {
  if (f.d == 1) return t;
  unsigned q = __umulhi(t, f.m);
  if (q * f.d > t) --q;
  return q;
}

// One Stockham pass over `nb` transforms of length n held in shared memory.
// Element i of transform b is at base[b*bs + i*es]. Ns = product of the radices of the
// previous passes. Twiddle table tw[q] = exp(-2 pi i q / n). Batch index runs fastest
// across threads.
template <int R>
__device__ __forceinline__ void fft_pass_r(const float2* __restrict__ in, float2* __restrict__ out, int n,
                                           int Ns, int nb, int es, int bs, const float2* __restrict__ tw,
                                           bool inv, int nb2, int bs2) {
  const int nbf = n / R;
  const int total = nb * nb2 * nbf;
  const int tws = n / (Ns * R);
  const FastDiv fnb = make_fdiv((unsigned)(nb * nb2)), fns = make_fdiv((unsigned)Ns), fb1 = make_fdiv((unsigned)nb);
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int j = (int)fdiv((unsigned)t, fnb);
    const int bb = t - j * (nb * nb2);
    const int b2 = (int)fdiv((unsigned)bb, fb1);
    const int b = bb - b2 * nb;
    const int jq = (int)fdiv((unsigned)j, fns);
    const int k = j - jq * Ns;
    const int boff = b * bs + b2 * bs2;
    const float2* src = in + boff;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[(j + r * nbf) * es];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        float2 w = tw[r * k * tws];
        if (inv) w.y = -w.y;
        v[r] = cmul(v[r], w);
      }
    }
    dft_reg<R>(v, inv, tw, n);
    const int idxD = jq * Ns * R + k;
    float2* dst = out + boff;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[(idxD + r * Ns) * es] = v[r];
  }
}

// Pass with a radix that has no register specialisation: one thread per output element.
__device__ __forceinline__ void fft_pass_any(const float2* __restrict__ in, float2* __restrict__ out, int n,
                                             int Ns, int R, int nb, int es, int bs,
                                             const float2* __restrict__ tw, bool inv, int nb2, int bs2) {
  const int nbf = n / R;
  const int total = nb * nb2 * n;
  const int tws = n / (Ns * R);
  const int st = n / R;
  const FastDiv fnb = make_fdiv((unsigned)(nb * nb2)), fnbf = make_fdiv((unsigned)nbf), fns = make_fdiv((unsigned)Ns),
                fb1 = make_fdiv((unsigned)nb);
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    const int rest = (int)fdiv((unsigned)t, fnb);
    const int bb = t - rest * (nb * nb2);
    const int b2 = (int)fdiv((unsigned)bb, fb1);
    const int b = bb - b2 * nb;
    const int s = (int)fdiv((unsigned)rest, fnbf);
    const int j = rest - s * nbf;
    const int jq = (int)fdiv((unsigned)j, fns);
    const int k = j - jq * Ns;
    const int boff = b * bs + b2 * bs2;
    const float2* src = in + boff;
    float2 acc = make_float2(0.f, 0.f);
    for (int r = 0; r < R; ++r) {
      float2 v = src[(j + r * nbf) * es];
      float2 w = tw[r * k * tws];
      float2 u = tw[((r * s) % R) * st];
      if (inv) {
        w.y = -w.y;
        u.y = -u.y;
      }
      acc = cadd(acc, cmul(cmul(v, w), u));
    }
    const int idxD = jq * Ns * R + k;
    out[boff + (idxD + s * Ns) * es] = acc;
  }
}

__device__ __forceinline__ void fft_pass(const float2* in, float2* out, int n, int Ns, int R, int nb, int es,
                                         int bs, const float2* tw, bool inv, int nb2, int bs2) {
  switch (R) {
    case 2: fft_pass_r<2>(in, out, n, Ns, nb, es, bs, tw, inv, nb2, bs2); break;
    case 3: fft_pass_r<3>(in, out, n, Ns, nb, es, bs, tw, inv, nb2, bs2); break;
    case 4: fft_pass_r<4>(in, out, n, Ns, nb, es, bs, tw, inv, nb2, bs2); break;
    case 5: fft_pass_r<5>(in, out, n, Ns, nb, es, bs, tw, inv, nb2, bs2); break;
    case 7: fft_pass_r<7>(in, out, n, Ns, nb, es, bs, tw, inv, nb2, bs2); break;
    case 8: fft_pass_r<8>(in, out, n, Ns, nb, es, bs, tw, inv, nb2, bs2); break;
    case 16: fft_pass_r<16>(in, out, n, Ns, nb, es, bs, tw, inv, nb2, bs2); break;
    default: fft_pass_any(in, out, n, Ns, R, nb, es, bs, tw, inv, nb2, bs2); break;
  }
}

// Full transform: passes ping-pong between *src and *dst (swapped after each pass); on
// return *src holds the result. A __syncthreads() follows every pass. Transforms are indexed
// by (b < nb, b2 < nb2) at b bs + b2 bs2 (nb2 > 1: blocks of slices transformed separately).
__device__ __forceinline__ void fft_run(float2** src, float2** dst, const FftPlan& p, int nb, int es, int bs,
                                        const float2* tw, bool inv, int nb2 = 1, int bs2 = 0) {
  int Ns = 1;
  for (int i = 0; i < p.np; ++i) {
    const int R = p.r[i];
    fft_pass(*src, *dst, p.n, Ns, R, nb, es, bs, tw, inv, nb2, bs2);
    __syncthreads();
    float2* t = *src;
    *src = *dst;
    *dst = t;
    Ns *= R;
  }
}

}  // namespace lps
#endif  // __CUDACC__
