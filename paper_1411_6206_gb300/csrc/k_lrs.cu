// Step (3) of Algorithm 1 (Sec. 3), the support-aware sparse update, one CTA per group of
// 8 x 8 in-plane tiles and all nc slices:
//   c = T(X_{k-1} - L_{k-1}) (orthonormal 2D Haar per slice, J levels),
//   c' = c on the prior support T^(t-1), soft(c, lambda_S) off it,
//   S_k = T^{-1}(c'); support bits [|c| > lambda_S].
// It needs neither the singular values nor W of the same iteration, so it runs concurrently
// with the eigen kernel; the reprojection L_k = (X_{k-1} - S_{k-1}) W of steps (1)-(2) is
// formed by the data-consistency kernel that consumes it. Partial sums for the objective
// (l1 off the support) and the support count are reduced per CTA in a fixed order.
//
// Wavelet coefficient layout: within a tile the 8 x 8 coefficient array holds, for every
// aligned 2^J x 2^J sub-block, that sub-block's own Mallat layout. Eight consecutive lanes
// hold the 64 coefficients of one (tile, slice), so four lanes give one 32-bit word of the
// bitmap.
//
// The 3D variant (Z3) is the tensor product of that 2D pyramid with the J-level 1D Haar along
// z on aligned blocks of 2^J slices: after the in-plane analysis every thread stores its row
// in shared memory, each thread then transforms the z columns of a (tile, z block, u, v) set,
// and the rows come back for the shrink; the synthesis runs the same passes in reverse. The
// slice z = 2^J bz + w of the bitmap then holds the coefficients of 1D position w (Mallat
// order inside the block) of z block bz.
#include "lps_internal.cuh"

#include <algorithm>

namespace lps {

// Thread layout: 8 consecutive lanes own one (tile, slice z); lane u holds row u of the
// slice's 8 x 8 tile as 8 complex registers v = 0..7. CTAs of 256 threads take
// TPC = floor(32 / nc) tiles by default (Geom::lrs_tpc overrides it).
__device__ __forceinline__ float2 shfl2(float2 v, int src) {
  return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// One analysis level l (1-based) of the orthonormal 2D Haar on every aligned B x B
// sub-block (B = 2^J) of the 8 x 8 tile, in place in the Mallat layout of each sub-block.
// A = B >> (l-1) is the edge of the current approximation region, H = A/2.
template <int J, int L>
__device__ __forceinline__ void haar_fwd_level(float2 (&r)[8], int u, int lane) {
  constexpr int B = 1 << J, A = B >> (L - 1), H = A / 2;
  const int su = u / B, ul = u - su * B;          // sub-block row, row inside it
  const bool act = ul < A;
  const int gi = ul < H ? ul : ul - H;            // group row
  const int s0 = (lane & ~7) + su * B + 2 * gi;   // source lanes (rows 2gi, 2gi+1)
  float2 e[8], o[8];
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    e[v] = shfl2(r[v], s0);
    o[v] = shfl2(r[v], s0 + 1);
  }
  if (!act) return;
  // x split: rows (2gi, 2gi+1) -> low (top half of the region) or high (bottom half)
  float2 row[8];
#pragma unroll
  for (int v = 0; v < 8; ++v) row[v] = ul < H ? cadd(e[v], o[v]) : csub(e[v], o[v]);
  // y split inside every sub-block column range, scaled 1/2 (two 1/sqrt(2) factors)
#pragma unroll
  for (int sv = 0; sv < 8 / B; ++sv) {
    float2 t[A];
#pragma unroll
    for (int q = 0; q < H; ++q) {
      t[q] = cscale(cadd(row[sv * B + 2 * q], row[sv * B + 2 * q + 1]), 0.5f);
      t[q + H] = cscale(csub(row[sv * B + 2 * q], row[sv * B + 2 * q + 1]), 0.5f);
    }
#pragma unroll
    for (int q = 0; q < A; ++q) r[sv * B + q] = t[q];
  }
}

template <int J, int L>
__device__ __forceinline__ void haar_inv_level(float2 (&r)[8], int u, int lane) {
  constexpr int B = 1 << J, A = B >> (L - 1), H = A / 2;
  const int su = u / B, ul = u - su * B;
  const bool act = ul < A;
  const int gi = ul >> 1;
  const int s_lo = (lane & ~7) + su * B + gi;      // approximation / x-low row
  const int s_hi = s_lo + H;                       // x-high row
  float2 lo[8], hi[8];
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    lo[v] = shfl2(r[v], s_lo);
    hi[v] = shfl2(r[v], s_hi);
  }
  if (!act) return;
  float2 row[8];
#pragma unroll
  for (int v = 0; v < 8; ++v) row[v] = (ul & 1) ? csub(lo[v], hi[v]) : cadd(lo[v], hi[v]);
#pragma unroll
  for (int sv = 0; sv < 8 / B; ++sv) {
    float2 t[A];
#pragma unroll
    for (int q = 0; q < H; ++q) {
      t[2 * q] = cscale(cadd(row[sv * B + q], row[sv * B + q + H]), 0.5f);
      t[2 * q + 1] = cscale(csub(row[sv * B + q], row[sv * B + q + H]), 0.5f);
    }
#pragma unroll
    for (int q = 0; q < A; ++q) r[sv * B + q] = t[q];
  }
}

template <int J>
__device__ __forceinline__ void haar_fwd(float2 (&r)[8], int u, int lane) {
  haar_fwd_level<J, 1>(r, u, lane);
  if constexpr (J >= 2) haar_fwd_level<J, 2>(r, u, lane);
  if constexpr (J >= 3) haar_fwd_level<J, 3>(r, u, lane);
}
template <int J>
__device__ __forceinline__ void haar_inv(float2 (&r)[8], int u, int lane) {
  if constexpr (J >= 3) haar_inv_level<J, 3>(r, u, lane);
  if constexpr (J >= 2) haar_inv_level<J, 2>(r, u, lane);
  haar_inv_level<J, 1>(r, u, lane);
}

// z pass of the 3D variant. zb holds one row of 8 complex per thread, row r at zb + 8r with
// element v at position v ^ ((r >> 1) & 7): the row stores of a half-warp (16 rows, one
// element each) and the column reads (consecutive (u, v)) hit 32 distinct banks.
__device__ __forceinline__ int zslot(int row, int v) { return row * 8 + (v ^ ((row >> 1) & 7)); }

__device__ __forceinline__ void zrow_store(float2* zb, int row, const float2 (&r)[8]) {
#pragma unroll
  for (int v = 0; v < 8; ++v) zb[zslot(row, v)] = r[v];
}
__device__ __forceinline__ void zrow_load(const float2* zb, int row, float2 (&r)[8]) {
#pragma unroll
  for (int v = 0; v < 8; ++v) r[v] = zb[zslot(row, v)];
}

// J-level 1D Haar along z (forward or inverse, Mallat order inside each aligned block of
// B = 2^J slices) on the columns (tile, z block, u, v) of zb; the columns are spread over the
// CTA's threads. Returns max |c| of the forward coefficients this thread produced (MAXC).
template <int J, bool INV, bool MAXC>
__device__ __forceinline__ float zpass(float2* zb, int nc, int tpc, int tid, int nthr) {
  constexpr int B = 1 << J;
  constexpr float r2 = 0.70710678118654752f;
  const int nzb = nc / B;
  const int ncol = tpc * nzb * 64;
  float mx = 0.f;
  for (int col = tid; col < ncol; col += nthr) {
    const int uv = col & 63, rest = col >> 6;
    const int tl = rest / nzb, bz = rest - tl * nzb;
    const int row0 = (tl * nc + bz * B) * 8 + (uv >> 3), v = uv & 7;
    float2 f[B];
#pragma unroll
    for (int w = 0; w < B; ++w) f[w] = zb[zslot(row0 + 8 * w, v)];
    if constexpr (!INV) {
#pragma unroll
      for (int l = 1; l <= J; ++l) {
        const int A = B >> (l - 1), H = A / 2;
        float2 t[B];
#pragma unroll
        for (int q = 0; q < B / 2; ++q) {
          if (q < H) {
            t[q] = cscale(cadd(f[2 * q], f[2 * q + 1]), r2);
            t[q + H] = cscale(csub(f[2 * q], f[2 * q + 1]), r2);
          }
        }
#pragma unroll
        for (int q = 0; q < B; ++q)
          if (q < A) f[q] = t[q];
      }
      if constexpr (MAXC) {
#pragma unroll
        for (int w = 0; w < B; ++w) mx = fmaxf(mx, sqrtf(cabs2(f[w])));
      }
    } else {
#pragma unroll
      for (int l = J; l >= 1; --l) {
        const int A = B >> (l - 1), H = A / 2;
        float2 t[B];
#pragma unroll
        for (int q = 0; q < B / 2; ++q) {
          if (q < H) {
            t[2 * q] = cscale(cadd(f[q], f[q + H]), r2);
            t[2 * q + 1] = cscale(csub(f[q], f[q + H]), r2);
          }
        }
#pragma unroll
        for (int q = 0; q < B; ++q)
          if (q < A) f[q] = t[q];
      }
    }
    if constexpr (!MAXC) {
#pragma unroll
      for (int w = 0; w < B; ++w) zb[zslot(row0 + 8 * w, v)] = f[w];
    }
  }
  return mx;
}

template <int J, bool Z3>
__global__ void __launch_bounds__(1024) k_lrs(const LrsArgs a) {
  const Geom& g = a.g;
  extern __shared__ __align__(16) unsigned char smem[];
  float* red = reinterpret_cast<float*>(smem);
  float2* zb = reinterpret_cast<float2*>(smem + 32 * sizeof(float));   // Z3: one row per thread
  const int nc = g.nz;   // slices per tile (every slice of the volume)
  const int tpc = g.lrs_tpc > 0 ? g.lrs_tpc : (32 / nc > 0 ? 32 / nc : 1);   // tiles per CTA

  const int tid = threadIdx.x, lane = tid & 31;
  const int u = tid & 7, grp = tid >> 3;
  const int tl = grp / nc, z = grp - tl * nc;
  const int nty = g.ny >> 3;
  const int tile = blockIdx.x * tpc + tl;
  const bool act = tl < tpc && tile < g.ntiles;
  const int tx = act ? tile / nty : 0, ty = act ? tile - (tile / nty) * nty : 0;
  const long long nxy = (long long)g.nx * g.ny;
  const long long rowoff = (long long)z * nxy + (long long)(tx * 8 + u) * g.ny + ty * 8;
  const bool maxonly = a.haar_max_only != 0;
  // this lane's 8 coefficients are bits [u*8, u*8+8) of the (z, tile) 64-bit group
  const long long wbase = ((long long)(z * (g.nx >> 3) + tx) * nty + ty) * 2;

  pdl_trigger();
  pdl_wait();   // X, L and the control block come from the preceding kernels
  // Every independent global load is issued up front: their latencies overlap.
  const int conv = a.ctrl->converged;
  // lambda_S is fixed with lambda_L by the eigen kernel of the first iteration, which may run
  // concurrently with this one; until then it is lambda_S_rel * max |T(X_0)| (the same value)
  const int lset = a.ctrl->lambdas_set;
  const float lamS_set = a.ctrl->lambda_S;
  const float hmax = __uint_as_float(a.ctrl->haar_max_bits);
  const int has_sup = a.persist->has_sup;
  const unsigned prior_word = (act && !maxonly) ? a.sup_prior[wbase + (u >> 2)] : 0u;
  float2 Xr[8], Lp[8];
#pragma unroll
  for (int v = 0; v < 8; ++v) Xr[v] = Lp[v] = make_float2(0.f, 0.f);
  if (act) {
    const float4* xs = reinterpret_cast<const float4*>(a.X + rowoff);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float4 q = xs[i];
      Xr[2 * i] = make_float2(q.x, q.y);
      Xr[2 * i + 1] = make_float2(q.z, q.w);
    }
    if (!maxonly) {
      const float4* ls = reinterpret_cast<const float4*>(a.L + rowoff);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float4 q = ls[i];
        Lp[2 * i] = make_float2(q.x, q.y);
        Lp[2 * i + 1] = make_float2(q.z, q.w);
      }
    }
  }
  if (conv) return;

  if (maxonly) {
    haar_fwd<J>(Xr, u, lane);
    float mx = 0.f;
    if constexpr (Z3) {
      zrow_store(zb, tid, Xr);
      __syncthreads();
      mx = zpass<J, false, true>(zb, nc, tpc, tid, blockDim.x);
    } else {
#pragma unroll
      for (int v = 0; v < 8; ++v) mx = fmaxf(mx, sqrtf(cabs2(Xr[v])));
    }
    mx = block_max(mx, red);
    if (tid == 0) atomicMax(&a.ctrl->haar_max_bits, __float_as_uint(mx));
    return;
  }
  const float lamS = lset ? lamS_set : (float)(a.lambda_S_rel * (double)hmax);

  // Sparse step on D = X - L_prev: Haar analysis, support-aware shrink, synthesis.
  float2 D[8];
#pragma unroll
  for (int v = 0; v < 8; ++v) D[v] = csub(Xr[v], Lp[v]);
  haar_fwd<J>(D, u, lane);
  if constexpr (Z3) {
    zrow_store(zb, tid, D);
    __syncthreads();
    zpass<J, false, false>(zb, nc, tpc, tid, blockDim.x);
    __syncthreads();
    zrow_load(zb, tid, D);
  }
  const unsigned keepbits = has_sup ? (prior_word >> ((u & 3) * 8)) & 0xffu : 0u;
  float l1 = 0.f;
  unsigned sbits = 0;
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    const float2 c = D[v];
    const float ab = sqrtf(cabs2(c));
    const bool keep = (keepbits >> v) & 1u;
    float2 cs = c;
    if (!keep) {
      cs = cscale(c, ab > lamS ? (ab - lamS) / ab : 0.f);
      l1 += ab > lamS ? ab - lamS : 0.f;
    }
    const bool bit = (a.support_rule == 0) ? (ab > lamS) : (cs.x != 0.f || cs.y != 0.f);
    sbits |= (unsigned)bit << v;
    D[v] = cs;
  }
  // gather the bytes of lanes u = 0..3 (word 0) and u = 4..7 (word 1)
  unsigned word = sbits << ((u & 3) * 8);
  word |= __shfl_xor_sync(0xffffffffu, word, 1);
  word |= __shfl_xor_sync(0xffffffffu, word, 2);
  if (act && (u & 3) == 0 && a.sup_out) a.sup_out[wbase + (u >> 2)] = word;
  const float cnt = (act && (u & 3) == 0) ? (float)__popc(word) : 0.f;
  if (!act) l1 = 0.f;
  if constexpr (Z3) {
    zrow_store(zb, tid, D);   // the same slots this thread loaded: no barrier needed before
    __syncthreads();
    zpass<J, true, false>(zb, nc, tpc, tid, blockDim.x);
    __syncthreads();
    zrow_load(zb, tid, D);
  }
  haar_inv<J>(D, u, lane);
  if (act) {
    float4* sd = reinterpret_cast<float4*>(a.S + rowoff);
#pragma unroll
    for (int i = 0; i < 4; ++i) sd[i] = make_float4(D[2 * i].x, D[2 * i].y, D[2 * i + 1].x, D[2 * i + 1].y);
  }
  float* part = a.lrs_part + (long long)blockIdx.x * 2;
  float r;
  r = block_sum(l1, red);
  if (tid == 0) part[0] = r;
  r = block_sum(cnt, red);
  if (tid == 0) part[1] = r;
}

// Partials of the Casorati Gram (X - S)^H (X - S) straight from global memory; used when
// the state is loaded from outside rather than produced by the data-consistency step. CTA p
// sums the planes x = p q .. p q + q - 1 (q = nx / nparts), so the eigen kernel finds the
// same number of partials as the data-consistency step leaves.
__global__ void __launch_bounds__(kThreads) k_gram_plane(const float2* X, const float2* S, Geom g,
                                                         float2* gram_part, int nparts) {
  extern __shared__ __align__(16) unsigned char smem[];
  float2* M = reinterpret_cast<float2*>(smem);   // [nz][nyp]
  const int ny = g.ny, nyp = g.nyp, nc = g.nc;
  const int q = g.nx / nparts;
  const long long nxy = (long long)g.nx * ny;
  float2* gp = gram_part + (long long)blockIdx.x * nc * nc;
  for (int x = blockIdx.x * q; x < (int)(blockIdx.x + 1) * q; ++x) {
    __syncthreads();
    for (int e = threadIdx.x; e < g.plane; e += kThreads) {
      const int z = e / ny, y = e - (e / ny) * ny;
      const long long gi = z * nxy + (long long)x * ny + y;
      M[z * nyp + y] = S ? csub(X[gi], S[gi]) : X[gi];
    }
    __syncthreads();
    const bool first = x == (int)blockIdx.x * q;
    // each thread owns its entries across the planes, so the running sums need no barrier;
    // column i holds slices i cs .. i cs + cs - 1
    for (int t = threadIdx.x; t < nc * nc; t += kThreads) {
      const int i = t / nc, j = t - (t / nc) * nc;
      if (i > j) continue;
      float sr = 0.f, si = 0.f;
      for (int s = 0; s < g.cs; ++s)
        for (int y = 0; y < ny; ++y) {
          const float2 u = M[(i * g.cs + s) * nyp + y], v = M[(j * g.cs + s) * nyp + y];
          sr = fmaf(u.x, v.x, fmaf(u.y, v.y, sr));
          si = fmaf(u.x, v.y, fmaf(-u.y, v.x, si));
        }
      if (!first) {
        const float2 o = gp[i * nc + j];
        sr += o.x;
        si += o.y;
      }
      if (i == j) si = 0.f;   // exactly real diagonal
      gp[i * nc + j] = make_float2(sr, si);
      if (i != j) gp[j * nc + i] = make_float2(sr, -si);
    }
  }
}

// recon = L + S, the reconstructed volume of Algorithm 1's output.
__global__ void k_combine(const float2* __restrict__ L, const float2* __restrict__ S, float2* __restrict__ out,
                          long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = cadd(L[i], S[i]);
}

__global__ void k_round_half(float2* __restrict__ c, __half2* __restrict__ h, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const __half2 v = __float22half2_rn(c[i]);
    h[i] = v;
    c[i] = __half22float2(v);
  }
}

cudaError_t launch_round_half(float2* c, __half2* h, long long n, cudaStream_t st) {
  const int blocks = (int)std::min<long long>((n + kThreads - 1) / kThreads, 152 * 16);
  k_round_half<<<blocks, kThreads, 0, st>>>(c, h, n);
  return cudaGetLastError();
}

cudaError_t launch_combine(const float2* L, const float2* S, float2* out, long long n, cudaStream_t st) {
  const int blocks = (int)std::min<long long>((n + kThreads - 1) / kThreads, 152LL * 8);
  k_combine<<<blocks, kThreads, 0, st>>>(L, S, out, n);
  return cudaGetLastError();
}

int lrs_tpc(const Geom& g) { return g.lrs_tpc > 0 ? g.lrs_tpc : std::max(1, 32 / g.nz); }

// Threads of one sparse-step CTA: 8 per (tile, slice), rounded up to whole warps (the
// Haar shuffles need full warps; lanes beyond the tiles are inactive).
int lrs_threads(const Geom& g) { return (8 * g.nz * lrs_tpc(g) + 31) / 32 * 32; }

static size_t lrs_smem(const Geom& g) {
  return 32 * sizeof(float) + (g.wz ? (size_t)lrs_threads(g) * 8 * sizeof(float2) : 0);
}

int lrs_blocks(const Geom& g) { return (g.ntiles + lrs_tpc(g) - 1) / lrs_tpc(g); }

template <int J, bool Z3>
static cudaError_t launch_lrs_j(const LrsArgs& a, cudaStream_t st) {
  const size_t smem = lrs_smem(a.g);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_lrs<J, Z3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = launch_pdl(k_lrs<J, Z3>, dim3(lrs_blocks(a.g)), dim3(lrs_threads(a.g)), smem, st, a);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_lrs(const LrsArgs& a, cudaStream_t st) {
  // the 3D variant needs whole z blocks (validated with the plan's parameters)
  if (a.g.wz && a.g.nz % (1 << a.g.J) != 0) return cudaErrorInvalidValue;
  if (lrs_threads(a.g) > 1024) return cudaErrorInvalidValue;
  switch (a.g.J * 2 + (a.g.wz ? 1 : 0)) {
    case 2: return launch_lrs_j<1, false>(a, st);
    case 3: return launch_lrs_j<1, true>(a, st);
    case 4: return launch_lrs_j<2, false>(a, st);
    case 5: return launch_lrs_j<2, true>(a, st);
    case 7: return launch_lrs_j<3, true>(a, st);
    default: return launch_lrs_j<3, false>(a, st);
  }
}

// End of a run of iterations: the sparse step alternates its outputs (S, support words,
// statistic partials) between two buffers by iteration, and the run may have stopped early
// on the relative-change rule. Buffer 1 holds the last completed iteration's outputs when
// the count of iterations completed in this run (iters_done - k0 + 1) is odd; copy them to
// buffer 0 then.
__global__ void k_settle(const DevCtrl* __restrict__ ctrl, int k0, float2* S0, const float2* __restrict__ S1,
                         long long n, uint32_t* sup0, const uint32_t* __restrict__ sup1, long long nw, float* part0,
                         const float* __restrict__ part1, int np) {
  pdl_wait();
  const int done = ctrl->iters_done - k0 + 1;   // iterations completed in this run
  if (done <= 0 || (done & 1) == 0) return;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  for (long long i = t0; i < n; i += stride) S0[i] = S1[i];
  for (long long i = t0; i < nw; i += stride) sup0[i] = sup1[i];
  for (long long i = t0; i < np; i += stride) part0[i] = part1[i];
}

cudaError_t launch_settle(const DevCtrl* ctrl, int k0, float2* S0, const float2* S1, long long n, uint32_t* sup0,
                          const uint32_t* sup1, long long nw, float* part0, const float* part1, int np,
                          cudaStream_t st) {
  const int blocks = (int)std::min<long long>((n + 255) / 256, 152LL * 4);
  k_settle<<<blocks, 256, 0, st>>>(ctrl, k0, S0, S1, n, sup0, sup1, nw, part0, part1, np);
  return cudaGetLastError();
}

// G = sum of the nparts partials, in partial order (one thread per entry).
__global__ void k_gram_sum(const float2* __restrict__ part, int nparts, int nn, float2* __restrict__ G) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nn) return;
  float2 s = make_float2(0.f, 0.f);
  for (int p = 0; p < nparts; ++p) s = cadd(s, part[(long long)p * nn + e]);
  G[e] = s;
}

cudaError_t launch_gram_sum(const float2* part, int nparts, int nc, float2* G, cudaStream_t st) {
  const int nn = nc * nc;
  k_gram_sum<<<(nn + 255) / 256, 256, 0, st>>>(part, nparts, nn, G);
  return cudaGetLastError();
}

// L[j][r] = sum_i (X - S)[i][r] W[i][j] in float32, one thread per pixel r (the stand-alone
// form of the reprojection that k_lrs fuses with the sparse step).
__global__ void k_reproj_f32(const float2* __restrict__ X, const float2* __restrict__ S,
                             const float2* __restrict__ W, float2* __restrict__ L, Geom g) {
  const long long nr = g.N / g.nc;   // rows of the Casorati matrix (voxels of a column)
  const int nc = g.nc;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < nr; r += (long long)gridDim.x * blockDim.x) {
    float2 m[kMaxNc];
#pragma unroll
    for (int i = 0; i < kMaxNc; ++i)
      m[i] = i < nc ? (S ? csub(X[i * nr + r], S[i * nr + r]) : X[i * nr + r]) : make_float2(0.f, 0.f);
    for (int j = 0; j < nc; ++j) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < kMaxNc; ++i) {
        if (i < nc) {
          const float2 w = W[i * nc + j];
          acc.x = fmaf(m[i].x, w.x, fmaf(-m[i].y, w.y, acc.x));
          acc.y = fmaf(m[i].x, w.y, fmaf(m[i].y, w.x, acc.y));
        }
      }
      L[j * nr + r] = acc;
    }
  }
}

cudaError_t launch_reproj_f32(const float2* X, const float2* S, const float2* W, float2* L, const Geom& g,
                              cudaStream_t st) {
  const long long nr = g.N / g.nc;
  const int blocks = (int)std::min<long long>((nr + 127) / 128, 152LL * 8);
  k_reproj_f32<<<blocks, 128, 0, st>>>(X, S, W, L, g);
  return cudaGetLastError();
}

cudaError_t launch_gram_plane(const float2* X, const float2* S, const Geom& g, float2* gram_part, int nparts,
                              cudaStream_t st) {
  if (nparts <= 0 || g.nx % nparts != 0) return cudaErrorInvalidValue;
  const size_t smem = (size_t)g.planeP * sizeof(float2);
  if (smem > 48 * 1024) {
    cudaError_t e =
        cudaFuncSetAttribute(k_gram_plane, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_gram_plane<<<nparts, kThreads, smem, st>>>(X, S, g, gram_part, nparts);
  return cudaGetLastError();
}

}  // namespace lps
