// Steps (1)-(3) of Algorithm 1 (Sec. 3) that touch the Casorati matrix, one CTA per
// 8 x 8 in-plane tile and all nc slice columns:
//   step (1)+(2) reprojection   L_new = (X - S) W,  W = V diag(sigma''/sigma) V^H
//                               (= U diag(sigma'') V^H of the thresholded SVD; W comes
//                               from the eigendecomposition kernel)
//   step (3) sparse update      c = T(X - L_prev) (orthonormal 2D Haar per slice, J levels),
//                               c' = c on the prior support T^(t-1), soft(c, lambda_S) off it,
//                               S_new = T^{-1}(c'); support bits [|c| > lambda_S].
// Partial sums for the objective (l1 off the support) and for the relative-change stopping
// rule are reduced per tile in a fixed order.
//
// Wavelet coefficient layout: within a tile the 8 x 8 coefficient array holds, for every
// aligned 2^J x 2^J sub-block, that sub-block's own Mallat layout. Thread t owns tile row
// (u, v) = ((t&63)>>3, t&7) of the slices z = (t>>6) + 4q, so a warp covers 32 consecutive
// coefficients of one slice and one ballot gives one 32-bit word of the bitmap.
#include "lps_internal.cuh"

#include <algorithm>

namespace lps {

constexpr int kNQ = kMaxNc / 4;   // slices per thread

// One Haar analysis level l (1-based) on D[z][64] for all nc slices, sub-block size B.
__device__ __forceinline__ void haar_level_fwd(float2* D, int nc, int B, int l) {
  const int a = B >> (l - 1), half = a >> 1;
  const int gdim = 8 >> l;                 // groups per tile edge at this level
  const int ng = gdim * gdim;
  const int tasks = nc * ng;
  float2 o[2][4];
  int base[2];
  int cnt = 0;
  for (int t = threadIdx.x; t < tasks; t += blockDim.x, ++cnt) {
    const int z = t / ng, gidx = t - (t / ng) * ng;
    const int gu = gidx / gdim, gv = gidx - (gidx / gdim) * gdim;
    const int su = gu / half, sv = gv / half, iu = gu - su * half, iv = gv - sv * half;
    const int ou = su * B, ov = sv * B;
    const float2* Dz = D + z * 64;
    const float2 p00 = Dz[(ou + 2 * iu) * 8 + ov + 2 * iv];
    const float2 p01 = Dz[(ou + 2 * iu) * 8 + ov + 2 * iv + 1];
    const float2 p10 = Dz[(ou + 2 * iu + 1) * 8 + ov + 2 * iv];
    const float2 p11 = Dz[(ou + 2 * iu + 1) * 8 + ov + 2 * iv + 1];
    const float2 s0 = cadd(p00, p01), d0 = csub(p00, p01);   // along y
    const float2 s1 = cadd(p10, p11), d1 = csub(p10, p11);
    o[cnt][0] = cscale(cadd(s0, s1), 0.5f);   // approximation
    o[cnt][1] = cscale(cadd(d0, d1), 0.5f);   // x-low / y-high
    o[cnt][2] = cscale(csub(s0, s1), 0.5f);   // x-high / y-low
    o[cnt][3] = cscale(csub(d0, d1), 0.5f);   // x-high / y-high
    base[cnt] = z * 64 + (ou + iu) * 8 + ov + iv;
  }
  __syncthreads();
  for (int i = 0; i < cnt; ++i) {
    float2* Dz = D + base[i];
    Dz[0] = o[i][0];
    Dz[half] = o[i][1];
    Dz[half * 8] = o[i][2];
    Dz[half * 8 + half] = o[i][3];
  }
  __syncthreads();
}

__device__ __forceinline__ void haar_level_inv(float2* D, int nc, int B, int l) {
  const int a = B >> (l - 1), half = a >> 1;
  const int gdim = 8 >> l;
  const int ng = gdim * gdim;
  const int tasks = nc * ng;
  float2 o[2][4];
  int base[2];
  int cnt = 0;
  for (int t = threadIdx.x; t < tasks; t += blockDim.x, ++cnt) {
    const int z = t / ng, gidx = t - (t / ng) * ng;
    const int gu = gidx / gdim, gv = gidx - (gidx / gdim) * gdim;
    const int su = gu / half, sv = gv / half, iu = gu - su * half, iv = gv - sv * half;
    const int ou = su * B, ov = sv * B;
    const float2* Dz = D + z * 64 + (ou + iu) * 8 + ov + iv;
    const float2 ll = Dz[0], hy = Dz[half], hx = Dz[half * 8], hh = Dz[half * 8 + half];
    const float2 s0 = cadd(ll, hx), s1 = csub(ll, hx);   // undo x split
    const float2 d0 = cadd(hy, hh), d1 = csub(hy, hh);
    o[cnt][0] = cscale(cadd(s0, d0), 0.5f);   // (2iu, 2iv)
    o[cnt][1] = cscale(csub(s0, d0), 0.5f);   // (2iu, 2iv+1)
    o[cnt][2] = cscale(cadd(s1, d1), 0.5f);   // (2iu+1, 2iv)
    o[cnt][3] = cscale(csub(s1, d1), 0.5f);   // (2iu+1, 2iv+1)
    base[cnt] = z * 64 + (ou + 2 * iu) * 8 + ov + 2 * iv;
  }
  __syncthreads();
  for (int i = 0; i < cnt; ++i) {
    float2* Dz = D + base[i];
    Dz[0] = o[i][0];
    Dz[1] = o[i][1];
    Dz[8] = o[i][2];
    Dz[9] = o[i][3];
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kThreads) k_lrs(const LrsArgs a) {
  const Geom& g = a.g;
  if (a.ctrl->converged) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int nc = g.nc, ncp = nc + 1;
  float2* Msh = reinterpret_cast<float2*>(smem);   // [64][ncp]
  float2* Dsh = Msh + 64 * ncp;                     // [nc][64]
  float2* Wsh = Dsh + nc * 64;                      // [nc][nc]
  float* red = reinterpret_cast<float*>(Wsh + nc * nc);

  const int tid = threadIdx.x;
  const int nty = g.ny >> 3;
  const int tile = blockIdx.x;
  const int tx = tile / nty, ty = tile - (tile / nty) * nty;
  const int row = tid & 63, zg = tid >> 6;
  const int u = row >> 3, v = row & 7;
  const long long nxy = (long long)g.nx * g.ny;
  const long long goff = (long long)(tx * 8 + u) * g.ny + ty * 8 + v;
  const int B = 1 << g.J;
  const bool maxonly = a.haar_max_only != 0;

  float2 Lp[kNQ], So[kNQ];
#pragma unroll
  for (int q = 0; q < kNQ; ++q) {
    const int z = zg + 4 * q;
    Lp[q] = So[q] = make_float2(0.f, 0.f);
    if (z < nc) {
      const long long gi = z * nxy + goff;
      const float2 Xv = a.X[gi];
      if (maxonly) {
        Dsh[z * 64 + row] = Xv;
      } else {
        const float2 Sv = a.S[gi], Lv = a.L[gi];
        Msh[row * ncp + z] = csub(Xv, Sv);
        Dsh[z * 64 + row] = csub(Xv, Lv);
        Lp[q] = Lv;
        So[q] = Sv;
      }
    }
  }
  if (!maxonly)
    for (int i = tid; i < nc * nc; i += kThreads) Wsh[i] = a.W[i];
  __syncthreads();
  for (int l = 1; l <= g.J; ++l) haar_level_fwd(Dsh, nc, B, l);

  if (maxonly) {
    float mx = 0.f;
    for (int i = tid; i < nc * 64; i += kThreads) mx = fmaxf(mx, sqrtf(cabs2(Dsh[i])));
    mx = block_max(mx, red);
    if (tid == 0) atomicMax(&a.ctrl->haar_max_bits, __float_as_uint(mx));
    return;
  }

  // Reprojection L_new[row][z] = sum_i M[row][i] W[i][z].
  float2 Ln[kNQ];
#pragma unroll
  for (int q = 0; q < kNQ; ++q) Ln[q] = make_float2(0.f, 0.f);
  for (int i = 0; i < nc; ++i) {
    const float2 mv = Msh[row * ncp + i];
#pragma unroll
    for (int q = 0; q < kNQ; ++q) {
      const int z = zg + 4 * q;
      if (z < nc) {
        const float2 w = Wsh[i * nc + z];
        Ln[q].x = fmaf(mv.x, w.x, fmaf(-mv.y, w.y, Ln[q].x));
        Ln[q].y = fmaf(mv.x, w.y, fmaf(mv.y, w.x, Ln[q].y));
      }
    }
  }

  // Support-aware shrink of the coefficients (thread: slices z, coefficient `row`).
  const float lamS = a.ctrl->lambda_S;
  const bool has_sup = a.persist->has_sup != 0;
  const int lane = tid & 31;
  float l1 = 0.f, cnt = 0.f;
#pragma unroll
  for (int q = 0; q < kNQ; ++q) {
    const int z = zg + 4 * q;
    if (z < nc) {   // uniform across the warp
      const long long word = ((long long)(z * (g.nx >> 3) + tx) * nty + ty) * 2 + (row >> 5);
      const float2 c = Dsh[z * 64 + row];
      const bool keep = has_sup && ((a.sup_prior[word] >> (row & 31)) & 1u);
      const float ab = sqrtf(cabs2(c));
      float2 cs = c;
      if (!keep) {
        const float f = ab > lamS ? (ab - lamS) / ab : 0.f;
        cs = cscale(c, f);
        l1 += ab > lamS ? ab - lamS : 0.f;
      }
      const bool bit = (a.support_rule == 0) ? (ab > lamS) : (cs.x != 0.f || cs.y != 0.f);
      const unsigned bal = __ballot_sync(0xffffffffu, bit);
      if (lane == 0) {
        if (a.sup_out) a.sup_out[word] = bal;
        cnt += (float)__popc(bal);
      }
      Dsh[z * 64 + row] = cs;
    }
  }
  __syncthreads();
  for (int l = g.J; l >= 1; --l) haar_level_inv(Dsh, nc, B, l);

  float dz2 = 0.f, z2 = 0.f;
#pragma unroll
  for (int q = 0; q < kNQ; ++q) {
    const int z = zg + 4 * q;
    if (z < nc) {
      const long long gi = z * nxy + goff;
      const float2 Sn = Dsh[z * 64 + row];
      a.S[gi] = Sn;
      a.L[gi] = Ln[q];
      const float2 Zo = cadd(Lp[q], So[q]);
      const float2 dZ = csub(cadd(Ln[q], Sn), Zo);
      dz2 += cabs2(dZ);
      z2 += cabs2(Zo);
    }
  }
  float* part = a.lrs_part + (long long)tile * 4;
  float r;
  r = block_sum(l1, red);
  if (tid == 0) part[0] = r;
  r = block_sum(dz2, red);
  if (tid == 0) part[1] = r;
  r = block_sum(z2, red);
  if (tid == 0) part[2] = r;
  r = block_sum(cnt, red);
  if (tid == 0) part[3] = r;
}

// Plane share of the Casorati Gram (X - S)^H (X - S) straight from global memory; used
// when the state is loaded from outside rather than produced by the data-consistency step.
__global__ void __launch_bounds__(kThreads) k_gram_plane(const float2* X, const float2* S, Geom g,
                                                         float2* gram_part) {
  extern __shared__ __align__(16) unsigned char smem[];
  float2* M = reinterpret_cast<float2*>(smem);   // [nz][nyp]
  const int x = blockIdx.x, ny = g.ny, nyp = g.nyp, nc = g.nc;
  const long long nxy = (long long)g.nx * ny;
  for (int e = threadIdx.x; e < g.plane; e += kThreads) {
    const int z = e / ny, y = e - (e / ny) * ny;
    const long long gi = z * nxy + (long long)x * ny + y;
    M[z * nyp + y] = csub(X[gi], S[gi]);
  }
  __syncthreads();
  float2* gp = gram_part + (long long)x * nc * nc;
  for (int t = threadIdx.x; t < nc * nc; t += kThreads) {
    const int i = t / nc, j = t - (t / nc) * nc;
    if (i > j) continue;
    float sr = 0.f, si = 0.f;
    for (int y = 0; y < ny; ++y) {
      const float2 p = M[i * nyp + y], q = M[j * nyp + y];
      sr = fmaf(p.x, q.x, fmaf(p.y, q.y, sr));
      si = fmaf(p.x, q.y, fmaf(-p.y, q.x, si));
    }
    gp[i * nc + j] = make_float2(sr, si);
    if (i != j) gp[j * nc + i] = make_float2(sr, -si);
  }
}

// recon = L + S, the reconstructed volume of Algorithm 1's output.
__global__ void k_combine(const float2* __restrict__ L, const float2* __restrict__ S, float2* __restrict__ out,
                          long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = cadd(L[i], S[i]);
}

cudaError_t launch_combine(const float2* L, const float2* S, float2* out, long long n, cudaStream_t st) {
  const int blocks = (int)std::min<long long>((n + kThreads - 1) / kThreads, 152LL * 8);
  k_combine<<<blocks, kThreads, 0, st>>>(L, S, out, n);
  return cudaGetLastError();
}

static size_t lrs_smem(const Geom& g) {
  return (size_t)(64 * (g.nc + 1) + g.nc * 64 + g.nc * g.nc) * sizeof(float2) + 32 * sizeof(float);
}

cudaError_t launch_lrs(const LrsArgs& a, cudaStream_t st) {
  const size_t smem = lrs_smem(a.g);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_lrs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_lrs<<<a.g.ntiles, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_gram_plane(const float2* X, const float2* S, const Geom& g, float2* gram_part,
                              cudaStream_t st) {
  const size_t smem = (size_t)g.planeP * sizeof(float2);
  if (smem > 48 * 1024) {
    cudaError_t e =
        cudaFuncSetAttribute(k_gram_plane, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_gram_plane<<<g.nx, kThreads, smem, st>>>(X, S, g, gram_part);
  return cudaGetLastError();
}

}  // namespace lps
