// Data-consistency step of Algorithm 1 (step 4, Sec. 3) and the acquisition operator of
// Sec. 2, one CTA per x-plane.
//
// E = M F C with F the orthonormal DFT over (z, x, y) and a mask M that does not depend on
// kx. The x-transform therefore commutes with M and cancels in E^H E; with the samples
// moved once to the hybrid space d' = F_x^H d (kernel k_xfft), step (4) becomes, for every
// x-plane independently,
//     X = Z - sum_c conj(C_c) F_yz^H [ M F_yz (C_c Z) - d'_c ],     Z = L + S,
// and ||E Z - d||^2 = sum over planes and coils of the masked residual energy.
// The epilogue forms the plane's share of the Casorati Gram (X - S)^H (X - S) used by
// the singular-value step of the next iteration.
//
// Per coil: coil plane staged by 1D TMA bulk copies (double buffered on mbarriers),
// elementwise multiply, y- and z-Stockham FFTs in shared memory, residual on the sampled
// lines, inverse FFTs, conjugate-coil accumulate in registers.
#include "lps_internal.cuh"

namespace lps {

// STAGE: coil planes staged in shared memory by TMA (1 CTA per SM for large planes); without,
// the coil values are read from global memory (L2) where they are used, which halves the
// shared memory so that two CTAs share an SM.
// HALF (direct reads of the update only): coil maps read as half-precision pairs
// (LPS_COILS_FP16), widened exactly to float32.
template <int EPT, int MODE, bool STAGE, bool HALF>
__global__ void __launch_bounds__(kThreads, STAGE ? 1 : 2) k_dc(const DcArgs a) {
  static_assert(!(HALF && (STAGE || MODE != kDcUpdate)), "half-precision coil maps: direct update only");
  const Geom& g = a.g;
  pdl_trigger();
  pdl_wait();
  if (a.ctrl && a.ctrl->converged) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int ny = g.ny, nz = g.nz, nx = g.nx, nyp = g.nyp;
  const int plane = g.plane;
  float2* bufA = reinterpret_cast<float2*>(smem);
  float2* bufB = bufA + g.planeP;
  float2* coilS0 = bufB + g.planeP;
  float2* coilS1 = coilS0 + (STAGE ? plane : 0);
  float2* twy = coilS1 + (STAGE ? plane : 0);
  float2* twz = twy + ny;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(twz + nz + ((ny + nz) & 1));
  float* red = reinterpret_cast<float*>(mbar + 2);
  float2* wsh = reinterpret_cast<float2*>(red + 32);   // [nz][nz] W of the iteration form

  const int tid = threadIdx.x;
  const int x = blockIdx.x;
  const long long xy = (long long)nx * ny;
  const int m = a.persist->nlines;
  int* errp = a.ctrl ? &a.ctrl->err : nullptr;

  for (int i = tid; i < ny; i += kThreads) twy[i] = a.tw_y[i];
  for (int i = tid; i < nz; i += kThreads) twz[i] = a.tw_z[i];
  if (STAGE && tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const unsigned coil_bytes = (unsigned)(ny * sizeof(float2));
  auto issue = [&](int c, float2* slot, uint64_t* bar) {
    mbar_arrive_expect_tx(bar, coil_bytes * nz);
    const float2* base = a.coils + (long long)c * g.N + (long long)x * ny;
    for (int z = 0; z < nz; ++z) bulk_g2s(slot + z * ny, base + z * xy, coil_bytes, bar);
  };
  // Thread 0 tracks which slots have a copy in flight (bit s) and their wait parity.
  unsigned inflight = 0;
  if (STAGE && tid == 0) {
    issue(0, coilS0, &mbar[0]);
    inflight |= 1u;
    if (g.ncoil > 1) {
      issue(1, coilS1, &mbar[1]);
      inflight |= 2u;
    }
  }

  // Element ownership for the elementwise phases: e = tid + k*kThreads.
  float2 Zr[EPT];
  float2 acc[EPT];
  int pe[EPT];    // padded offset z*nyp + y
  int go[EPT];    // offset z*nx*ny + y of the element in a coil plane starting at x*ny
  float dz2 = 0.f, z2 = 0.f;   // ||Z_k - Z_{k-1}||^2 and ||Z_{k-1}||^2
  const bool iter_form = MODE == kDcUpdate && (a.W != nullptr || a.Lpre != nullptr);
  // Every per-element global load is issued first, so that their latencies overlap: S_k,
  // X_{k-1}, S_{k-1} and L_{k-1} of the iteration form give M_{k-1} (into bufA), and
  // S_k - Z_{k-1} is kept for the change statistic.
  float2 Dz[EPT];
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int e = tid + k * kThreads;
    acc[k] = make_float2(0.f, 0.f);
    Zr[k] = Dz[k] = make_float2(0.f, 0.f);
    pe[k] = -1;
    go[k] = 0;
    if (e < plane) {
      const int z = e / ny, y = e - (e / ny) * ny;
      pe[k] = z * nyp + y;
      go[k] = (int)(z * xy) + y;
      const long long gi = (long long)z * xy + (long long)x * ny + y;
      if (iter_form) {
        Zr[k] = a.S[gi];
        const float2 Sp = a.Sprev[gi];
        const float2 Zo = cadd(a.Lbuf[gi], Sp);
        if (a.W) bufA[pe[k]] = csub(a.X[gi], Sp);
        Dz[k] = csub(Zr[k], Zo);
        z2 += cabs2(Zo);
      } else if (MODE != kDcAdjoint) {
        float2 v = a.L[gi];
        if (MODE == kDcUpdate && a.S) v = cadd(v, a.S[gi]);
        Zr[k] = v;
      }
    }
  }
  if (iter_form && a.W) {
    // Steps (1)-(2) completed here: L_k = (X_{k-1} - S_{k-1}) W over the plane's columns,
    // one pixel column and 4 output slices per task, into bufB.
    for (int i = tid; i < nz * nz; i += kThreads) wsh[i] = a.W[i];
    __syncthreads();
    const int nzb = (nz + 3) / 4;
    for (int task = tid; task < ny * nzb; task += kThreads) {
      const int y = task % ny, zb = (task / ny) * 4;
      float2 o[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) o[j] = make_float2(0.f, 0.f);
      for (int i = 0; i < nz; ++i) {
        const float2 mv = bufA[i * nyp + y];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (zb + j < nz) {
            const float2 w = wsh[i * nz + zb + j];
            o[j].x = fmaf(mv.x, w.x, fmaf(-mv.y, w.y, o[j].x));
            o[j].y = fmaf(mv.x, w.y, fmaf(mv.y, w.x, o[j].y));
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (zb + j < nz) bufB[(zb + j) * nyp + y] = o[j];
    }
    __syncthreads();
  }
  if (iter_form) {
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      if (pe[k] < 0) continue;
      const int e = tid + k * kThreads;
      const int z = e / ny, y = e - (e / ny) * ny;
      const long long gi = (long long)z * xy + (long long)x * ny + y;
      const float2 Lk = a.W ? bufB[pe[k]] : a.Lpre[gi];
      Zr[k] = cadd(Lk, Zr[k]);
      a.Lbuf[gi] = Lk;
      dz2 += cabs2(cadd(Lk, Dz[k]));
    }
  }
  if (iter_form && a.W) __syncthreads();   // bufA and bufB are the FFT buffers of the coil loop

  const float sc = g.scale_yz;
  float resid = 0.f;
  for (int c = 0; c < g.ncoil; ++c) {
    const int s = c & 1;
    float2* coil = s ? coilS1 : coilS0;
    const float2* gcoil = a.coils + (long long)c * g.N + (long long)x * ny;   // without staging
    const __half2* hcoil = HALF ? a.coils_h + (long long)c * g.N + (long long)x * ny : nullptr;
    auto gc = [&](int k) -> float2 { return HALF ? __half22float2(__ldg(hcoil + go[k])) : __ldg(gcoil + go[k]); };
    if (STAGE) {
      const bool bad = !mbar_wait_bounded(&mbar[s], (c >> 1) & 1, errp);
      if (__syncthreads_or(bad)) {
        // Give up on this plane; first let the other slot's copy (if any) land.
        if (tid == 0 && (inflight & (2u >> s))) mbar_wait_bounded(&mbar[s ^ 1], ((c + 1) >> 1) & 1, nullptr);
        return;
      }
      if (tid == 0) inflight &= ~(1u << s);
    }
    float2* src = bufA;
    float2* dst = bufB;
    const float2* dh = a.dhyb + ((long long)x * g.ncoil + c) * g.mpad;
    if (MODE != kDcAdjoint) {
      // P = scale * C_c * Z, then the forward transform over y (rows) and z (columns).
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int e = tid + k * kThreads;
        if (e < plane) src[pe[k]] = cscale(cmul(STAGE ? coil[e] : gc(k), Zr[k]), sc);
      }
      __syncthreads();
      fft_run(&src, &dst, g.py, nz, 1, nyp, twy, false);
      if (g.fft_z) fft_run(&src, &dst, g.pz, ny, nyp, 1, twz, false);
      if (MODE == kDcForward) {
        float2* ho = a.hyb_out + ((long long)x * g.ncoil + c) * g.mpad;
        for (int l = tid; l < m; l += kThreads) ho[l] = src[a.lines[l]];
        __syncthreads();
        if (STAGE && tid == 0 && c + 2 < g.ncoil) {
          fence_proxy_async();
          issue(c + 2, coil, &mbar[s]);
          inflight |= 1u << s;
        }
        continue;
      }
    }
    // Residual on the sampled lines: R = M (F C Z) - d' (update) or the samples (adjoint).
#pragma unroll
    for (int k = 0; k < EPT; ++k)
      if (pe[k] >= 0) dst[pe[k]] = make_float2(0.f, 0.f);
    __syncthreads();
    for (int l = tid; l < m; l += kThreads) {
      const int p = a.lines[l];
      float2 r;
      if (MODE == kDcAdjoint) {
        r = dh[l];
      } else {
        r = csub(src[p], dh[l]);
        resid = fmaf(r.x, r.x, fmaf(r.y, r.y, resid));
      }
      dst[p] = r;
    }
    __syncthreads();
    {
      float2* t = src;
      src = dst;
      dst = t;
    }
    if (g.fft_z) fft_run(&src, &dst, g.pz, ny, nyp, 1, twz, true);
    fft_run(&src, &dst, g.py, nz, 1, nyp, twy, true);
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int e = tid + k * kThreads;
      if (e < plane) {
        const float2 r = src[pe[k]];
        const float2 cc = STAGE ? coil[e] : gc(k);
        const float2 v = cmulc(cc, r);   // conj(C) * r
        acc[k].x = fmaf(v.x, sc, acc[k].x);
        acc[k].y = fmaf(v.y, sc, acc[k].y);
      }
    }
    __syncthreads();
    if (STAGE && tid == 0 && c + 2 < g.ncoil) {
      fence_proxy_async();
      issue(c + 2, coil, &mbar[s]);
      inflight |= 1u << s;
    }
  }
  if (MODE == kDcForward) return;

  // X = Z - E^H(E Z - d)  (update) or X_0 = E^H d (adjoint); then M = X - S into bufA.
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int e = tid + k * kThreads;
    if (e < plane) {
      const int z = e / ny, y = e - (e / ny) * ny;
      const long long gi = (long long)z * xy + (long long)x * ny + y;
      float2 Xv, Mv;
      if (MODE == kDcUpdate) {
        Xv = csub(Zr[k], acc[k]);
        if (a.recon) a.recon[gi] = Zr[k];
        Mv = a.S ? csub(Xv, a.S[gi]) : Xv;
      } else {
        Xv = acc[k];
        Mv = Xv;
        if (a.L_out) a.L_out[gi] = Xv;
        if (a.S_out) a.S_out[gi] = make_float2(0.f, 0.f);
      }
      a.X[gi] = Xv;
      bufA[pe[k]] = Mv;
    }
  }
  __syncthreads();
  if (a.gram_part) {
    // Plane share of G = M^H M: G[i][j] = sum_y conj(M[i][y]) M[j][y], columns i, j = slices.
    const int nc = g.nc;
    float2* gp = a.gram_part + (long long)x * nc * nc;
    for (int t = tid; t < nc * nc; t += kThreads) {
      const int i = t / nc, j = t - (t / nc) * nc;
      if (i > j) continue;
      const float2* ri = bufA + i * nyp;
      const float2* rj = bufA + j * nyp;
      float sr = 0.f, si = 0.f;
      for (int y = 0; y < ny; ++y) {
        const float2 u = ri[y], v = rj[y];
        sr = fmaf(u.x, v.x, fmaf(u.y, v.y, sr));
        si = fmaf(u.x, v.y, fmaf(-u.y, v.x, si));
      }
      gp[i * nc + j] = make_float2(sr, si);
      if (i != j) gp[j * nc + i] = make_float2(sr, -si);
    }
  }
  if (MODE == kDcUpdate && a.dc_part) {
    const float r2 = block_sum(resid, red);
    const float d2 = block_sum(dz2, red);
    const float o2 = block_sum(z2, red);
    if (tid == 0) reinterpret_cast<float4*>(a.dc_part)[x] = make_float4(r2, d2, o2, 0.f);
  }
}

int dc_ept(const Geom& g) {
  const int need = (g.plane + kThreads - 1) / kThreads;
  if (need <= 1) return 1;
  if (need <= 2) return 2;
  if (need <= 4) return 4;
  if (need <= 8) return 8;
  if (need <= 16) return 16;
  if (need <= 24) return 24;
  return -1;
}

size_t dc_smem_bytes(const Geom& g) {
  size_t b = 0;
  b += 2 * (size_t)g.planeP * sizeof(float2);
  if (!g.dc_direct) b += 2 * (size_t)g.plane * sizeof(float2);   // staged coil planes
  b += (size_t)(g.ny + g.nz + ((g.ny + g.nz) & 1)) * sizeof(float2);
  b += 2 * sizeof(uint64_t);
  b += 32 * sizeof(float);
  b += (size_t)g.nz * g.nz * sizeof(float2);   // W of the iteration form
  return b;
}

template <int EPT, int MODE, bool STAGE, bool HALF>
static cudaError_t launch_dc_t(const DcArgs& a, cudaStream_t st) {
  const size_t smem = dc_smem_bytes(a.g);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_dc<EPT, MODE, STAGE, HALF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)227 * 1024);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  cudaError_t e = launch_pdl(k_dc<EPT, MODE, STAGE, HALF>, dim3(a.g.nx), dim3(kThreads), smem, st, a);
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <int MODE, bool STAGE, bool HALF>
static cudaError_t launch_dc_m(const DcArgs& a, cudaStream_t st) {
  switch (dc_ept(a.g)) {
    case 1: return launch_dc_t<1, MODE, STAGE, HALF>(a, st);
    case 2: return launch_dc_t<2, MODE, STAGE, HALF>(a, st);
    case 4: return launch_dc_t<4, MODE, STAGE, HALF>(a, st);
    case 8: return launch_dc_t<8, MODE, STAGE, HALF>(a, st);
    case 16: return launch_dc_t<16, MODE, STAGE, HALF>(a, st);
    case 24: return launch_dc_t<24, MODE, STAGE, HALF>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

// Staged coil planes are copied in float32 (the rounded maps); the direct variant of the update
// reads the half-precision copy when the plan keeps one.
template <int MODE>
static cudaError_t launch_dc_s(const DcArgs& a, cudaStream_t st) {
  if (!a.g.dc_direct) return launch_dc_m<MODE, true, false>(a, st);
  if constexpr (MODE == kDcUpdate) {
    if (a.coils_h) return launch_dc_m<MODE, false, true>(a, st);
  }
  return launch_dc_m<MODE, false, false>(a, st);
}

cudaError_t launch_dc_fixed(const DcArgs& a, int mode, cudaStream_t st);

// The update of a 128 x 16 plane goes to the register-transform kernel (k_dc_reg) unless the
// plan selected another variant; other plane sizes with a compile-time specialisation go to
// k_dc_fixed; the rest to k_dc.
cudaError_t launch_dc(const DcArgs& a, int mode, cudaStream_t st) {
  if (mode == kDcUpdate) {
    const cudaError_t er = launch_dc_reg(a, st);
    if (er != cudaErrorNotSupported) return er;
  }
  const cudaError_t ef = launch_dc_fixed(a, mode, st);
  if (ef != cudaErrorNotSupported) return ef;
  if (dc_smem_bytes(a.g) > 227 * 1024) return cudaErrorInvalidValue;
  switch (mode) {
    case kDcUpdate: return launch_dc_s<kDcUpdate>(a, st);
    case kDcAdjoint: return launch_dc_s<kDcAdjoint>(a, st);
    case kDcForward: return launch_dc_s<kDcForward>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lps
