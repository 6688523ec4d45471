// Tensor-core (tcgen05) forms of the two dense contractions of Algorithm 1 (Sec. 3), used by
// the precision modes (LPS_TF32_REFINE, LPS_BF16_REFINE):
//   - the Casorati Gram G = M^H M, M = X - S (the input of the SVT, step (1)), and
//   - the low-rank reprojection L = M W, W = V diag(sigma''/sigma) V^H (steps (1)-(2)).
//
// Complex products as real ones. With M = a + i b and Q = [a | b] (N_r x 2n),
//   Q^T Q = [[a'a, a'b], [b'a, b'b]]  gives  Re G = a'a + b'b,  Im G = a'b - b'a,
//   [Re L | Im L] = Q [[Re W, Im W], [-Im W, Re W]].
// One refinement step: every float32 operand x is split x = hi + lo, hi = round(x) and
// lo = round(x - hi) in the operand type, and the products keep hi hi + hi lo + lo hi; the
// dropped lo lo term and the rounding of lo are about 2^-16 (bf16, 8-bit significand) or
// 2^-21 (tf32, 11 bits) relative to |x|^2. Accumulation is float32 in tensor memory.
//
// Layout of the shared-memory operands: K-major, no swizzle. A core matrix is 8 rows x 16
// bytes (rows 16 B apart); the core matrix of row group g and K chunk c sits at byte
// (g * KC + c) * 128, so adjacent K chunks are 128 B apart (leading byte offset) and adjacent
// row groups KC * 128 B apart (stride byte offset). Each MMA consumes two K chunks (32 bytes
// of K); the next one starts 256 B further.
//
// One thread issues the MMAs; tcgen05.commit arrives on an mbarrier when they are done. Every
// wait on an mbarrier is bounded; on a timeout the kernel records kErrTimeout, waits once more
// (bounded) for its MMAs, frees its tensor memory and returns.
#include "lps_internal.cuh"

#include <cuda_bf16.h>

namespace lps {

namespace {

constexpr int kTcThreads = 128;       // thread t owns pixel t of a tile and tensor-memory lane t
constexpr int kTcTile = 128;          // pixels per tile
constexpr uint32_t kTmemCols = 64;    // accumulator columns (N <= 64)

struct Bf16Op {
  using T = uint16_t;
  static constexpr int kBytes = 2;
  static constexpr uint32_t kFmt = 1;   // instruction-descriptor format code (kind::f16, BF16)
  __device__ static __forceinline__ void split(float x, T& hi, T& lo) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(l);
  }
};

struct Tf32Op {
  using T = uint32_t;
  static constexpr int kBytes = 4;
  static constexpr uint32_t kFmt = 2;   // kind::tf32
  __device__ static __forceinline__ void split(float x, T& hi, T& lo) {
    uint32_t h, l;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(x - __uint_as_float(h)));
    hi = h;
    lo = l;
  }
};

// Instruction descriptor: D float32 (bits 4-5 = 1), A and B format (bits 7-9, 10-12), both
// K-major (bits 15, 16 = 0), N >> 3 (bits 17-22), M >> 4 (bits 24-28).
__host__ __device__ constexpr uint32_t instr_desc(uint32_t fmt, int M, int N) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Shared-memory matrix descriptor: start address >> 4 (bits 0-13), leading byte offset >> 4
// (16-29), stride byte offset >> 4 (32-45), descriptor version 1 (bits 46-48), no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

template <uint32_t FMT>
__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  if constexpr (FMT == 1) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
  }
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Whole warp: allocate kTmemCols columns; the address lands in *slot.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(kTmemCols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTmemCols) : "memory");
}

// 16 consecutive float32 columns of this thread's lane; the wait is tied to the registers.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&out)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15])
               :
               : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) out[i] = __uint_as_float(r[i]);
}

// Byte offset of element (row, k) in a K-major core-matrix layout with kc chunks per row group.
template <class Op>
__device__ __forceinline__ uint32_t core_off(int row, int k, int kc) {
  constexpr int CE = 16 / Op::kBytes;   // elements per 16-byte core-matrix row
  return (uint32_t)(((row >> 3) * kc + k / CE) * 128 + (row & 7) * 16 + (k % CE) * Op::kBytes);
}

template <class Op>
__device__ __forceinline__ void st_op(unsigned char* base, uint32_t off, typename Op::T v) {
  *reinterpret_cast<typename Op::T*>(base + off) = v;
}

__device__ __forceinline__ int round_up(int v, int m) { return (v + m - 1) / m * m; }

}  // namespace

// ---- Gram: G_p = sum over this CTA's tiles of M^H M -------------------------------------
// A = [Qh^T; Ql^T] (4n rows, zero-padded to 128) times B = Qh (the first N rows of the same
// buffer) gives D = [Qh^T Qh; Ql^T Qh]; G_real = D_top + D_bot + D_bot^T. Two stages of
// kTcTile pixels: threads fill one while the tensor core reads the other.
template <class Op>
__global__ void __launch_bounds__(kTcThreads, 1) k_gram_tc(const GramTcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  constexpr int CE = 16 / Op::kBytes;
  constexpr int KC = kTcTile / CE;               // K chunks per stage
  constexpr uint32_t SB = 16u * KC * 128u;       // stage bytes (128 rows)
  constexpr int KI = 2 * CE;                     // K per MMA
  unsigned char* stage[2] = {smem, smem + SB};
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * SB);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  int* flag = reinterpret_cast<int*>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = a.g.nc;
  const int N = round_up(2 * n, 16);
  const long long nr = (long long)a.g.nx * a.g.ny;
  const int ntiles = (int)((nr + kTcTile - 1) / kTcTile);
  int* errp = a.ctrl ? &a.ctrl->err : nullptr;

  if (warp == 0) tmem_alloc(tslot);
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
    *flag = 0;
  }
  for (uint32_t i = tid * 16; i < 2 * SB; i += kTcThreads * 16)
    *reinterpret_cast<uint4*>(smem + i) = make_uint4(0u, 0u, 0u, 0u);
  pdl_trigger();
  pdl_wait();   // X and S come from the preceding kernels
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = instr_desc(Op::kFmt, 128, N);
  const int conv = a.ctrl ? a.ctrl->converged : 0;

  int it = 0;
  bool bad = false;
  for (int tile = blockIdx.x; tile < ntiles && !conv; tile += gridDim.x, ++it) {
    const int s = it & 1;
    // the stage's previous MMAs (iteration it - 2) must be done before it is overwritten
    if (it >= 2 && !mbar_wait_bounded(&bar[s], (unsigned)(((it >> 1) - 1) & 1), errp)) bad = true;
    if (__syncthreads_or(bad)) {
      bad = true;
      break;
    }
    const long long r = (long long)tile * kTcTile + tid;
    float2 m[kMaxNc];
#pragma unroll
    for (int z = 0; z < kMaxNc; ++z) {
      m[z] = make_float2(0.f, 0.f);
      if (z < n && r < nr) {
        const float2 x = a.X[z * nr + r];
        m[z] = a.S ? csub(x, a.S[z * nr + r]) : x;
      }
    }
    unsigned char* st = stage[s];
#pragma unroll
    for (int z = 0; z < kMaxNc; ++z) {
      if (z < n) {
        typename Op::T rh, rl, ih, il;
        Op::split(m[z].x, rh, rl);
        Op::split(m[z].y, ih, il);
        st_op<Op>(st, core_off<Op>(z, tid, KC), rh);
        st_op<Op>(st, core_off<Op>(n + z, tid, KC), ih);
        st_op<Op>(st, core_off<Op>(2 * n + z, tid, KC), rl);
        st_op<Op>(st, core_off<Op>(3 * n + z, tid, KC), il);
      }
    }
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t base = smem_u32(st);
#pragma unroll 1
      for (int k = 0; k < kTcTile / KI; ++k) {
        const uint64_t d = smem_desc(base + k * 256, 128, KC * 128);
        tc_mma<Op::kFmt>(tmem, d, d, idesc, (it > 0 || k > 0) ? 1u : 0u);
      }
      tc_commit(&bar[s]);
    }
  }
  // drain: the last commit covers every MMA issued before it
  if (it > 0) {
    const int l = it - 1;
    if (!mbar_wait_bounded(&bar[l & 1], (unsigned)((l >> 1) & 1), errp)) bad = true;
  }
  tc_fence_after();
  bad = __syncthreads_or(bad);

  // epilogue: D rows -> shared memory (stage 0 is free now), then this CTA's partial
  float* Dsh = reinterpret_cast<float*>(smem);   // [128][N + 1]
  const int ldd = N + 1;
  if (!bad && it > 0) {
    const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      tmem_ld16(lane_addr + c0, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) Dsh[(warp * 32 + lane) * ldd + c0 + j] = v[j];
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    tmem_dealloc(tmem);
  }
  if (bad) return;
  float2* gp = a.gram_part + (long long)blockIdx.x * n * n;
  auto greal = [&](int p, int q) {   // (Qh^T Qh + Ql^T Qh + Qh^T Ql)[p][q]
    return Dsh[p * ldd + q] + Dsh[(2 * n + p) * ldd + q] + Dsh[(2 * n + q) * ldd + p];
  };
  for (int e = tid; e < n * n; e += kTcThreads) {
    const int i = e / n, j = e - (e / n) * n;
    if (i > j) continue;
    float2 v = make_float2(0.f, 0.f);
    if (it > 0) {
      v.x = greal(i, j) + greal(n + i, n + j);
      v.y = (i == j) ? 0.f : greal(i, n + j) - greal(n + i, j);
    }
    gp[i * n + j] = v;
    gp[j * n + i] = cconj(v);
  }
}

// ---- reprojection: L = M W for 128-pixel tiles ------------------------------------------
// A = [Mh | Mh | Ml] (128 pixels x 6n), B = [Wh; Wl; Wh] (6n x 2n): D = Mh Wh + Mh Wl + Ml Wh.
template <class Op>
__global__ void __launch_bounds__(kTcThreads, 1) k_reproj_tc(const ReprojTcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  constexpr int CE = 16 / Op::kBytes;
  constexpr int KI = 2 * CE;
  const int n = a.g.nc;
  const int N = round_up(2 * n, 16);
  const int K = round_up(6 * n, KI);
  const int KC = K / CE;
  const uint32_t BB = (uint32_t)(N / 8) * KC * 128u;   // B bytes
  const uint32_t AB = 16u * KC * 128u;                 // A bytes
  unsigned char* Bs = smem;
  unsigned char* As = smem + BB;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + BB + AB);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  const long long nr = (long long)a.g.nx * a.g.ny;
  const int ntiles = (int)((nr + kTcTile - 1) / kTcTile);
  int* errp = a.ctrl ? &a.ctrl->err : nullptr;

  if (warp == 0) tmem_alloc(tslot);
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    fence_mbar_init();
  }
  for (uint32_t i = tid * 16; i < BB + AB; i += kTcThreads * 16)
    *reinterpret_cast<uint4*>(smem + i) = make_uint4(0u, 0u, 0u, 0u);
  pdl_trigger();
  pdl_wait();   // W, X and S come from the preceding kernels
  const int conv = a.ctrl ? a.ctrl->converged : 0;
  __syncthreads();
  // B^T rows j (output column), K index seg * 2n + k: Wr[k][j] split into hi / lo
  for (int e = tid; e < 4 * n * n; e += kTcThreads) {
    const int k = e / (2 * n), j = e - (e / (2 * n)) * (2 * n);
    const int kk = k < n ? k : k - n, jj = j < n ? j : j - n;
    const float2 w = a.W[kk * n + jj];
    const float wr = (k < n) == (j < n) ? w.x : (k < n ? w.y : -w.y);
    typename Op::T hi, lo;
    Op::split(wr, hi, lo);
    st_op<Op>(Bs, core_off<Op>(j, k, KC), hi);
    st_op<Op>(Bs, core_off<Op>(j, 2 * n + k, KC), lo);
    st_op<Op>(Bs, core_off<Op>(j, 4 * n + k, KC), hi);
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = instr_desc(Op::kFmt, 128, N);
  const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);

  int it = 0;
  bool bad = false;
  for (int tile = blockIdx.x; tile < ntiles && !conv; tile += gridDim.x, ++it) {
    const long long r = (long long)tile * kTcTile + tid;
    float2 m[kMaxNc];
#pragma unroll
    for (int z = 0; z < kMaxNc; ++z) {
      m[z] = make_float2(0.f, 0.f);
      if (z < n && r < nr) m[z] = a.S ? csub(a.X[z * nr + r], a.S[z * nr + r]) : a.X[z * nr + r];
    }
#pragma unroll
    for (int z = 0; z < kMaxNc; ++z) {
      if (z < n) {
        typename Op::T rh, rl, ih, il;
        Op::split(m[z].x, rh, rl);
        Op::split(m[z].y, ih, il);
        st_op<Op>(As, core_off<Op>(tid, z, KC), rh);
        st_op<Op>(As, core_off<Op>(tid, n + z, KC), ih);
        st_op<Op>(As, core_off<Op>(tid, 2 * n + z, KC), rh);
        st_op<Op>(As, core_off<Op>(tid, 3 * n + z, KC), ih);
        st_op<Op>(As, core_off<Op>(tid, 4 * n + z, KC), rl);
        st_op<Op>(As, core_off<Op>(tid, 5 * n + z, KC), il);
      }
    }
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t abase = smem_u32(As), bbase = smem_u32(Bs);
#pragma unroll 1
      for (int k = 0; k < K / KI; ++k)
        tc_mma<Op::kFmt>(tmem, smem_desc(abase + k * 256, 128, KC * 128), smem_desc(bbase + k * 256, 128, KC * 128),
                         idesc, k > 0 ? 1u : 0u);
      tc_commit(&bar[0]);
    }
    if (!mbar_wait_bounded(&bar[0], (unsigned)(it & 1), errp)) bad = true;
    tc_fence_after();
    if (__syncthreads_or(bad)) {
      bad = true;
      break;
    }
    // D row of this pixel: columns j < n are Re L[j], n <= j < 2n are Im L[j - n]
    float* Lf = reinterpret_cast<float*>(a.Lnew);
    for (int c0 = 0; c0 < N; c0 += 16) {
      float t[16];
      tmem_ld16(lane_addr + c0, t);
      if (r < nr) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int j = c0 + q;
          if (j < 2 * n) {
            const int z = j < n ? j : j - n;
            Lf[2 * (z * nr + r) + (j < n ? 0 : 1)] = t[q];
          }
        }
      }
    }
    // tensor-memory reads and the A tile are done before the next tile's MMAs
    tc_fence_before();
    __syncthreads();
  }
  if (bad) mbar_wait_bounded(&bar[0], (unsigned)(it & 1), nullptr);   // the MMAs of the failed tile
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    tmem_dealloc(tmem);
  }
}

// ---- host side --------------------------------------------------------------------------
int gram_tc_parts(const Geom& g) {
  const long long nr = (long long)g.nx * g.ny;
  const int ntiles = (int)((nr + kTcTile - 1) / kTcTile);
  return ntiles < 148 ? ntiles : 148;
}

size_t gram_tc_smem(int precision) {
  const int bytes = precision == kPrecBf16 ? 2 : 4;
  const size_t sb = 16u * (kTcTile / (16 / bytes)) * 128u;
  return 2 * sb + 64;
}

size_t reproj_tc_smem(const Geom& g, int precision) {
  const int bytes = precision == kPrecBf16 ? 2 : 4;
  const int ce = 16 / bytes, ki = 2 * ce;
  const int n = g.nc;
  const int N = (2 * n + 15) / 16 * 16;
  const int K = (6 * n + ki - 1) / ki * ki;
  const int kc = K / ce;
  return (size_t)(N / 8) * kc * 128 + 16u * kc * 128 + 64;
}

template <class Op>
static cudaError_t launch_gram_op(const GramTcArgs& a, int precision, cudaStream_t st) {
  const size_t smem = gram_tc_smem(precision);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_gram_tc<Op>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  cudaError_t e = launch_pdl(k_gram_tc<Op>, dim3(gram_tc_parts(a.g)), dim3(kTcThreads), smem, st, a);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_gram_tc(const GramTcArgs& a, int precision, cudaStream_t st) {
  if (a.g.nc > kMaxNc || 4 * a.g.nc > 128) return cudaErrorInvalidValue;
  if (precision == kPrecBf16) return launch_gram_op<Bf16Op>(a, precision, st);
  if (precision == kPrecTf32) return launch_gram_op<Tf32Op>(a, precision, st);
  return cudaErrorInvalidValue;
}

template <class Op>
static cudaError_t launch_reproj_op(const ReprojTcArgs& a, int precision, cudaStream_t st) {
  const size_t smem = reproj_tc_smem(a.g, precision);
  static size_t set_for = 0;
  if (set_for < smem) {
    cudaError_t e = cudaFuncSetAttribute(k_reproj_tc<Op>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    set_for = smem;
  }
  const long long nr = (long long)a.g.nx * a.g.ny;
  const int ntiles = (int)((nr + kTcTile - 1) / kTcTile);
  const int grid = ntiles < 148 ? ntiles : 148;
  cudaError_t e = launch_pdl(k_reproj_tc<Op>, dim3(grid), dim3(kTcThreads), smem, st, a);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_reproj_tc(const ReprojTcArgs& a, int precision, cudaStream_t st) {
  if (a.g.nc > kMaxNc) return cudaErrorInvalidValue;
  if (precision == kPrecBf16) return launch_reproj_op<Bf16Op>(a, precision, st);
  if (precision == kPrecTf32) return launch_reproj_op<Tf32Op>(a, precision, st);
  return cudaErrorInvalidValue;
}

}  // namespace lps
