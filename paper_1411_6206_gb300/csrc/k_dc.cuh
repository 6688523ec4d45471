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
//
// Planes of ny = 16 Q (Q = 4..10) and even nz up to 32 run the coil loop of the update on
// register transforms (dc_rt_coils) instead of the shared-memory Stockham passes.
#pragma once

#include "dft_reg.cuh"
#include "lps_internal.cuh"

namespace lps {

// ---- register-transform coil loop (planes of ny = 16 Q by nz = NZ) -------------------------
//
// Per coil, three phases with two CTA barriers:
//  row phase:    16 lanes per row z, lane l holding y = 16 q + l (q < Q). P = scale C_c Z, the
//                Q-point DFT over q in registers, twiddles W_ny^(l k1), then the 16-point DFT
//                across the lanes (radix-2 decimation in frequency, shuffles): lane l ends with
//                ky = k1 + Q bitrev4(l), stored at l (Q|1) + k1 of the row's frequency slots.
//  column phase: one thread per ky, the nz-point DFT over z in registers, the residual on
//                the sampled (kz, ky) (line numbers from a per-row bitmap and its prefix
//                counts), the inverse nz-point DFT.
//  row phase:    the inverse of the first (decimation in time across the lanes from the
//                bit-reversed order, conjugate twiddles, inverse Q-point DFT), then
//                sums += scale conj(C_c) r.
// The coil maps of the next coil and the samples d'_c are copied to shared memory with
// cp.async while a coil is processed; each thread copies the map elements that its own row
// tasks read, so only the samples need the barrier.
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ float2 shfl_xor2(float2 v, int m) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

// 16-point DFT across the lanes of each half-warp, element-wise over v[0..Q): decimation in
// frequency, natural order in, lane l out holding index bitrev4(l). w16, w8, w4 are this lane's
// roots W_16^(l mod 8), W_8^(l mod 4), W_4^(l mod 2) (used by the lanes of the upper halves).
template <int Q>
__device__ __forceinline__ void xlane_fwd(float2 (&v)[Q], int l, float2 w16, float2 w8, float2 w4) {
  const float2 ws[3] = {w16, w8, w4};
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int h = 8 >> s;
    const bool bot = (l & h) != 0;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      const float2 p = shfl_xor2(v[k], h);
      if (s < 3)
        v[k] = bot ? cmul(csub(p, v[k]), ws[s < 3 ? s : 0]) : cadd(v[k], p);
      else
        v[k] = bot ? csub(p, v[k]) : cadd(v[k], p);
    }
  }
}
// Its inverse without the 1/16: bit-reversed order in, natural order out, conjugate roots.
template <int Q>
__device__ __forceinline__ void xlane_inv(float2 (&v)[Q], int l, float2 w16, float2 w8, float2 w4) {
  const float2 ws[3] = {cconj(w4), cconj(w8), cconj(w16)};
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int h = 1 << s;
    const bool bot = (l & h) != 0;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      const float2 p = shfl_xor2(v[k], h);
      if (s == 0) {
        v[k] = bot ? csub(p, v[k]) : cadd(v[k], p);
      } else {
        const float2 w = ws[s > 0 ? s - 1 : 0];
        v[k] = bot ? csub(p, cmul(w, v[k])) : cadd(v[k], cmul(w, p));
      }
    }
  }
}

// Threads of a k_dc CTA: 512 for the register-transform loop of planes with nz >= 20 (one row
// task per thread, a thread pair per z column), else kThreads.
__host__ __device__ constexpr int dc_threads(int rtz, int rtq) { return (rtq > 0 && rtz >= 20) ? 512 : kThreads; }

// Shared memory of the register-transform loop, from the start of the iteration-form W
// region (which it reuses): frequency rows, two coil-map stages, the samples, the mask
// bitmap and its prefix counts.
__host__ __device__ constexpr int rt_ps(int Q) { return 16 * (Q | 1); }
// mpad: the samples' staging slots (complex elements).
__host__ __device__ inline size_t rt_region_bytes(int nz, int ny, int mpad) {
  const int Q = ny / 16, WB = (ny + 31) / 32;
  const size_t sf = (size_t)nz * rt_ps(Q) > (size_t)nz * nz ? (size_t)nz * rt_ps(Q) : (size_t)nz * nz;
  return (sf + 2 * (size_t)nz * ny + (size_t)mpad) * sizeof(float2) + 2 * (size_t)nz * WB * sizeof(int);
}

// One z column split over a thread pair (h = 0, 1): thread h holds the samples z = 2m + h,
// transforms them (H = NZ/2 points), and one radix-2 step across the pair leaves it holding
// kz = k + h H. The inverse mirrors it (thread h ends with z = 2m + h again).
template <int NZ, bool INV>
__device__ __forceinline__ void zpair_dft(float2 (&v)[NZ / 2], int h) {
  constexpr int H = NZ / 2;
  if constexpr (!INV) {
    dftr::dft<H, false>(v);
#pragma unroll
    for (int k = 0; k < H; ++k) {
      const float2 o = h ? dftr::rot<NZ, false>(v[k], k) : v[k];
      const float2 p = shfl_xor2(o, 1);
      v[k] = h ? csub(p, o) : cadd(o, p);
    }
  } else {
#pragma unroll
    for (int k = 0; k < H; ++k) {
      const float2 p = shfl_xor2(v[k], 1);
      v[k] = h ? dftr::rot<NZ, true>(csub(p, v[k]), k) : cadd(v[k], p);
    }
    dftr::dft<H, true>(v);
  }
}

template <int NZ, int Q, int NTH>
__device__ __forceinline__ float dc_rt_coils(const DcArgs& a, const float2* __restrict__ zbuf,
                                             float2* __restrict__ abuf, const float2* __restrict__ twy,
                                             float2* region, int x, int m) {
  constexpr int L = 16, QP = Q | 1, PS = L * QP, NY = L * Q, WB = (NY + 31) / 32;
  constexpr int NT = NZ * L, RT = (NT + NTH - 1) / NTH;
  constexpr bool PAIR = NZ >= 20;   // z columns on thread pairs
  static_assert(!PAIR || (NZ % 2 == 0 && 2 * NY <= NTH), "thread pairs per column");
  static_assert(NT % 32 == 0, "whole warps of row tasks");
  constexpr int SF = NZ * PS > NZ * NZ ? NZ * PS : NZ * NZ;
  const Geom& g = a.g;
  float2* Sf = region;
  float2* stg0 = Sf + SF;
  float2* stg1 = stg0 + NZ * NY;
  float2* dsm = stg1 + NZ * NY;
  // the coil's samples are staged in shared memory when the frame's lines fit the slots the
  // launch provided, else read from L2
  const bool stage_d = m <= g.dc_rt_dsm;
  unsigned* rbits = reinterpret_cast<unsigned*>(dsm + g.dc_rt_dsm);
  int* rpre = reinterpret_cast<int*>(rbits + NZ * WB);
  const int tid = threadIdx.x, l = tid & 15;
  const int nyp = g.nyp;
  const long long xy = (long long)g.nx * NY;
  const float sc = g.scale_yz;

  // mask bitmap: bit ky of word (kz, ky / 32); rpre = line number of the word's first bit
  // (lines are numbered in raster order of (kz, ky))
  for (int i = tid; i < NZ * WB; i += NTH) rbits[i] = 0u;
  __syncthreads();
  for (int i = tid; i < m; i += NTH) {
    const int p = a.lines[i];
    const int kz = p / nyp, ky = p - (p / nyp) * nyp;
    atomicOr(&rbits[kz * WB + (ky >> 5)], 1u << (ky & 31));
  }
  __syncthreads();
  if (tid < 32) {
    constexpr int NW = NZ * WB, PER = (NW + 31) / 32;
    int cnt = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int i = tid * PER + j;
      cnt += i < NW ? __popc(rbits[i]) : 0;
    }
    int inc = cnt;   // inclusive scan over the lanes
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, inc, o);
      if (tid >= o) inc += t;
    }
    int run = inc - cnt;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int i = tid * PER + j;
      if (i < NW) {
        rpre[i] = run;
        run += __popc(rbits[i]);
      }
    }
  }
  // this lane's twiddles: W_ny^(l k1), and the cross-lane roots (W_16^j = tw_y[j Q])
  float2 tq[Q];
#pragma unroll
  for (int k = 0; k < Q; ++k) tq[k] = twy[l * k];
  const float2 w16 = twy[(l & 7) * Q], w8 = twy[(l & 3) * 2 * Q], w4 = twy[(l & 1) * 4 * Q];

  auto issue_stage = [&](int c, float2* stg) {
    const float2* base = a.coils + (long long)c * g.N + (long long)x * NY;
#pragma unroll
    for (int r = 0; r < RT; ++r) {
      const int t = tid + r * NTH;
      if (t < NT) {
        const int z = t >> 4;
#pragma unroll
        for (int q = 0; q < Q; ++q) cp_async8(stg + z * NY + L * q + l, base + z * xy + L * q + l);
      }
    }
  };
  issue_stage(0, stg0);
  cp_async_commit();
  float resid = 0.f;
  for (int c = 0; c < g.ncoil; ++c) {
    const float2* stg = (c & 1) ? stg1 : stg0;
    const float2* dh = a.dhyb + ((long long)x * g.ncoil + c) * g.mpad;
    // LPS_DATA_FP16: the half pairs are loaded into registers here and widened into the
    // staging slots after the row phase (their latency hidden behind it); otherwise cp.async
    // copies the float32 samples. Frames with more lines than slots read the rounded float32
    // copy from L2.
    constexpr int kHalfPer = 8;
    const bool half_stage = stage_d && a.dhyb_h != nullptr && m <= kHalfPer * NTH;
    __half2 hv[kHalfPer];
    if (half_stage) {
      const __half2* dhh = a.dhyb_h + ((long long)x * g.ncoil + c) * g.mpad;
#pragma unroll
      for (int u = 0; u < kHalfPer; ++u) {
        const int i = tid + u * NTH;
        hv[u] = i < m ? dhh[i] : __half2{};
      }
    } else if (stage_d) {
      for (int i = tid; i < m; i += NTH) cp_async8(dsm + i, dh + i);
    }
    const float2* dsrc = stage_d ? dsm : dh;
    cp_async_commit();
    if (c + 1 < g.ncoil) issue_stage(c + 1, (c & 1) ? stg0 : stg1);
    cp_async_commit();
    cp_async_wait<2>();   // this thread's map elements of coil c
    // row phase, forward
#pragma unroll 1
    for (int r = 0; r < RT; ++r) {
      const int t = tid + r * NTH;
      if (t < NT) {
        const int z = t >> 4;
        float2 v[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const int y = L * q + l;
          v[q] = cscale(cmul(stg[z * NY + y], zbuf[z * nyp + y]), sc);
        }
        dftr::dft<Q, false>(v);
#pragma unroll
        for (int k = 1; k < Q; ++k) v[k] = cmul(v[k], tq[k]);
        xlane_fwd<Q>(v, l, w16, w8, w4);
#pragma unroll
        for (int k = 0; k < Q; ++k) Sf[z * PS + l * QP + k] = v[k];
      }
    }
    if (half_stage) {
#pragma unroll
      for (int u = 0; u < kHalfPer; ++u) {
        const int i = tid + u * NTH;
        if (i < m) dsm[i] = __half22float2(hv[u]);
      }
    }
    cp_async_wait<1>();   // the samples of coil c (this thread's share)
    __syncthreads();
    // column phase: z transform, residual on the sampled lines, inverse z transform
    if constexpr (!PAIR) {
      for (int ky = tid; ky < NY; ky += NTH) {
        const int k2 = ky / Q, k1 = ky - k2 * Q;
        const int off = (int)(__brev((unsigned)k2) >> 28) * QP + k1;
        float2 v[NZ];
#pragma unroll
        for (int z = 0; z < NZ; ++z) v[z] = Sf[z * PS + off];
        if (g.fft_z) dftr::dft<NZ, false>(v);
        const int wi = ky >> 5;
        const unsigned bit = ky & 31, below = (1u << bit) - 1u;
#pragma unroll
        for (int kz = 0; kz < NZ; ++kz) {
          const unsigned bits = rbits[kz * WB + wi];
          if ((bits >> bit) & 1u) {
            const int line = rpre[kz * WB + wi] + __popc(bits & below);
            const float2 r = csub(v[kz], dsrc[line]);
            resid = fmaf(r.x, r.x, fmaf(r.y, r.y, resid));
            v[kz] = r;
          } else {
            v[kz] = make_float2(0.f, 0.f);
          }
        }
        if (g.fft_z) dftr::dft<NZ, true>(v);
#pragma unroll
        for (int z = 0; z < NZ; ++z) Sf[z * PS + off] = v[z];
      }
    } else if (tid < 2 * NY) {   // whole warps (2 NY = 32 Q)
      constexpr int H = NZ / 2;
      const int ky = tid >> 1, h = tid & 1;
      const int k2 = ky / Q, k1 = ky - k2 * Q;
      const int off = (int)(__brev((unsigned)k2) >> 28) * QP + k1;
      float2 v[H];
#pragma unroll
      for (int m2 = 0; m2 < H; ++m2) v[m2] = Sf[(2 * m2 + h) * PS + off];
      const bool fz = g.fft_z != 0;
      if (fz) zpair_dft<NZ, false>(v, h);
      const int wi = ky >> 5;
      const unsigned bit = ky & 31, below = (1u << bit) - 1u;
#pragma unroll
      for (int k = 0; k < H; ++k) {
        // frequency kz = k + h H after the transform; slice 2k + h without it
        const int kz = fz ? k + h * H : 2 * k + h;
        const unsigned bits = rbits[kz * WB + wi];
        if ((bits >> bit) & 1u) {
          const int line = rpre[kz * WB + wi] + __popc(bits & below);
          const float2 r = csub(v[k], dsrc[line]);
          resid = fmaf(r.x, r.x, fmaf(r.y, r.y, resid));
          v[k] = r;
        } else {
          v[k] = make_float2(0.f, 0.f);
        }
      }
      if (fz) zpair_dft<NZ, true>(v, h);
#pragma unroll
      for (int m2 = 0; m2 < H; ++m2) Sf[(2 * m2 + h) * PS + off] = v[m2];
    }
    __syncthreads();
    // row phase, inverse, and the conjugate-coil sum
#pragma unroll 1
    for (int r = 0; r < RT; ++r) {
      const int t = tid + r * NTH;
      if (t < NT) {
        const int z = t >> 4;
        float2 v[Q];
#pragma unroll
        for (int k = 0; k < Q; ++k) v[k] = Sf[z * PS + l * QP + k];
        xlane_inv<Q>(v, l, w16, w8, w4);
#pragma unroll
        for (int k = 1; k < Q; ++k) v[k] = cmul(v[k], cconj(tq[k]));
        dftr::dft<Q, true>(v);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const int y = L * q + l;
          const float2 cv = cmulc(stg[z * NY + y], v[q]);   // conj(C) r
          float2& s = abuf[z * nyp + y];
          s = make_float2(fmaf(cv.x, sc, s.x), fmaf(cv.y, sc, s.y));
        }
      }
    }
  }
  cp_async_wait<0>();
  return resid;
}


// STAGE: coil planes staged in shared memory by TMA (1 CTA per SM for large planes); without,
// the coil values are read from global memory (L2) where they are used, which halves the
// shared memory so that two CTAs share an SM.
// HALF (direct reads of the update only): coil maps read as half-precision pairs
// (LPS_COILS_FP16), widened exactly to float32.
// RTZ, RTQ > 0: the coil loop of the update runs on register transforms (dc_rt_coils) for
// planes of ny = 16 RTQ by nz = RTZ.
// The work of one x-plane x (the body of k_dc; also run by the persistent batch kernel).
template <int EPT, int MODE, bool STAGE, bool HALF, int RTZ = 0, int RTQ = 0>
__device__ __forceinline__ void dc_plane(const DcArgs& a, const int x) {
  constexpr int NTH = dc_threads(RTZ, RTQ);
  static_assert(!(HALF && (STAGE || MODE != kDcUpdate)), "half-precision coil maps: direct update only");
  static_assert(RTQ == 0 || (MODE == kDcUpdate && !STAGE && !HALF), "register transforms: direct float32 update only");
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
  float* red = reinterpret_cast<float*>(mbar + 3);   // mbar[2]: the stall test hook's barrier
  float2* wsh = reinterpret_cast<float2*>(red + 32);   // [nz][nz] W of the iteration form

  const int tid = threadIdx.x;
  const long long xy = (long long)nx * ny;
  const int m = a.persist->nlines;
  int* errp = a.ctrl ? &a.ctrl->err : a.err_word;

  for (int i = tid; i < ny; i += NTH) twy[i] = a.tw_y[i];
  for (int i = tid; i < g.zn; i += NTH) twz[i] = a.tw_z[i];
  if (STAGE && tid == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    mbar_init(&mbar[2], 1);   // never arrived on: the stall test hook waits on it
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

  // Element ownership for the elementwise phases: e = tid + k*NTH.
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
    const int e = tid + k * NTH;
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
    // Casorati column i is slices i cs .. i cs + cs - 1: L[j cs + s] = sum_i M[i cs + s] W[i][j]
    const int nc = g.nc, cs = g.cs;
    for (int i = tid; i < nc * nc; i += NTH) wsh[i] = a.W[i];
    __syncthreads();
    const int ncb = (nc + 3) / 4;
    for (int task = tid; task < ny * cs * ncb; task += NTH) {
      const int y = task % ny, r = task / ny, s = r % cs, jb = (r / cs) * 4;
      float2 o[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) o[j] = make_float2(0.f, 0.f);
      for (int i = 0; i < nc; ++i) {
        const float2 mv = bufA[(i * cs + s) * nyp + y];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (jb + j < nc) {
            const float2 w = wsh[i * nc + jb + j];
            o[j].x = fmaf(mv.x, w.x, fmaf(-mv.y, w.y, o[j].x));
            o[j].y = fmaf(mv.x, w.y, fmaf(mv.y, w.x, o[j].y));
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (jb + j < nc) bufB[((jb + j) * cs + s) * nyp + y] = o[j];
    }
    __syncthreads();
  }
  if (iter_form) {
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      if (pe[k] < 0) continue;
      const int e = tid + k * NTH;
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
  if constexpr (RTQ > 0) {
    // Z into bufA and zero sums into bufB ([z][nyp]); the coil loop leaves
    // sum_c scale conj(C_c) F^H (M F (scale C_c Z) - d'_c) in bufB.
#pragma unroll
    for (int k = 0; k < EPT; ++k)
      if (pe[k] >= 0) {
        bufA[pe[k]] = Zr[k];
        bufB[pe[k]] = make_float2(0.f, 0.f);
      }
    __syncthreads();
    resid = dc_rt_coils<RTZ, RTQ, NTH>(a, bufA, bufB, twy, wsh, x, m);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int e = tid + k * NTH;
      const int z = e / ny, y = e - (e / ny) * ny;
      const bool in = e < plane;
      pe[k] = in ? z * nyp + y : -1;
      Zr[k] = in ? bufA[pe[k]] : make_float2(0.f, 0.f);
      acc[k] = in ? bufB[pe[k]] : make_float2(0.f, 0.f);
    }
  } else {
  for (int c = 0; c < g.ncoil; ++c) {
    const int s = c & 1;
    float2* coil = s ? coilS1 : coilS0;
    const float2* gcoil = a.coils + (long long)c * g.N + (long long)x * ny;   // without staging
    const __half2* hcoil = HALF ? a.coils_h + (long long)c * g.N + (long long)x * ny : nullptr;
    auto gc = [&](int k) -> float2 { return HALF ? __half22float2(__ldg(hcoil + go[k])) : __ldg(gcoil + go[k]); };
    if (STAGE) {
      // test hook: the first coil waits on mbar[2], which nothing completes, for stall_polls
      // polls, so that the timeout path below runs
      const bool stall = c == 0 && a.stall_polls > 0;
      const bool bad = stall ? !mbar_wait_bounded(&mbar[2], 0, errp, a.stall_polls)
                             : !mbar_wait_bounded(&mbar[s], (c >> 1) & 1, errp);
      if (__syncthreads_or(bad)) {
        // Give up on this plane; first let the copies still in flight land (normal budget).
        if (tid == 0) {
          if (stall) {
            if (inflight & 1u) mbar_wait_bounded(&mbar[0], 0, nullptr);
            if (inflight & 2u) mbar_wait_bounded(&mbar[1], 0, nullptr);
          } else if (inflight & (2u >> s)) {
            mbar_wait_bounded(&mbar[s ^ 1], ((c + 1) >> 1) & 1, nullptr);
          }
        }
        return;
      }
      if (tid == 0) inflight &= ~(1u << s);
    }
    float2* src = bufA;
    float2* dst = bufB;
    const float2* dh = a.dhyb + ((long long)x * g.ncoil + c) * g.mpad;   // the rounded copy with LPS_DATA_FP16
    if (MODE != kDcAdjoint) {
      // P = scale * C_c * Z, then the forward transform over y (rows) and z (columns).
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int e = tid + k * NTH;
        if (e < plane) src[pe[k]] = cscale(cmul(STAGE ? coil[e] : gc(k), Zr[k]), sc);
      }
      __syncthreads();
      fft_run(&src, &dst, g.py, nz, 1, nyp, twy, false);
      if (g.fft_z) fft_run(&src, &dst, g.pz, ny, nyp, 1, twz, false, nz / g.zn, g.zn * nyp);
      if (MODE == kDcForward) {
        float2* ho = a.hyb_out + ((long long)x * g.ncoil + c) * g.mpad;
        for (int l = tid; l < m; l += NTH) ho[l] = src[a.lines[l]];
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
    for (int l = tid; l < m; l += NTH) {
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
    if (g.fft_z) fft_run(&src, &dst, g.pz, ny, nyp, 1, twz, true, nz / g.zn, g.zn * nyp);
    fft_run(&src, &dst, g.py, nz, 1, nyp, twy, true);
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int e = tid + k * NTH;
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
  }
  if (MODE == kDcForward) return;

  // X = Z - E^H(E Z - d)  (update) or X_0 = E^H d (adjoint); then M = X - S into bufA.
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int e = tid + k * NTH;
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
    // Plane share of G = M^H M: G[i][j] = sum over the column's slices s and y of
    // conj(M[i cs + s][y]) M[j cs + s][y] (columns i, j; cs = 1: the slices).
    const int nc = g.nc, cs = g.cs;
    float2* gp = a.gram_part + (long long)x * nc * nc;
    for (int t = tid; t < nc * nc; t += NTH) {
      const int i = t / nc, j = t - (t / nc) * nc;
      if (i > j) continue;
      float sr = 0.f, si = 0.f;
      for (int s = 0; s < cs; ++s) {
        const float2* ri = bufA + (i * cs + s) * nyp;
        const float2* rj = bufA + (j * cs + s) * nyp;
        for (int y = 0; y < ny; ++y) {
          const float2 u = ri[y], v = rj[y];
          sr = fmaf(u.x, v.x, fmaf(u.y, v.y, sr));
          si = fmaf(u.x, v.y, fmaf(-u.y, v.x, si));
        }
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


template <int EPT, int MODE, bool STAGE, bool HALF, int RTZ = 0, int RTQ = 0>
__global__ void __launch_bounds__(dc_threads(RTZ, RTQ), (STAGE || RTZ >= 20) ? 1 : 2) k_dc(const DcArgs a) {
  dc_plane<EPT, MODE, STAGE, HALF, RTZ, RTQ>(a, blockIdx.x);
}

// Elements per thread of the runtime-sized kernel's elementwise phases, rounded up to the
// compiled values (1, 2, 4, 8, 16, 24; -1: plane too large).
__host__ __device__ constexpr int dc_ept_of(int plane, int nth = kThreads) {
  return (plane + nth - 1) / nth <= 1   ? 1
         : (plane + nth - 1) / nth <= 2 ? 2
         : (plane + nth - 1) / nth <= 4 ? 4
         : (plane + nth - 1) / nth <= 8 ? 8
         : (plane + nth - 1) / nth <= 16 ? 16
         : (plane + nth - 1) / nth <= 24 ? 24
                                        : -1;
}

template <int EPT, int MODE, bool STAGE, bool HALF, int RTZ = 0, int RTQ = 0>
static cudaError_t launch_dc_t(const DcArgs& a, size_t smem, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_dc<EPT, MODE, STAGE, HALF, RTZ, RTQ>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)227 * 1024);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  cudaError_t e = launch_pdl(k_dc<EPT, MODE, STAGE, HALF, RTZ, RTQ>, dim3(a.g.nx), dim3(dc_threads(RTZ, RTQ)), smem,
                             st, a);
  return e != cudaSuccess ? e : cudaGetLastError();
}

// Register-transform update for one nz (instantiated per nz in its own translation unit).
template <int NZ>
cudaError_t launch_dc_rt_nz(const DcArgs& a, size_t smem, cudaStream_t st) {
#define LPS_RT_CASE(Q)                                                                     \
  case Q:                                                                                  \
    return launch_dc_t<dc_ept_of(16 * Q * NZ, dc_threads(NZ, Q)), kDcUpdate, false, false, NZ, Q>(a, smem, st);
  switch (a.g.ny / 16) {
    LPS_RT_CASE(4)
    LPS_RT_CASE(5)
    LPS_RT_CASE(6)
    LPS_RT_CASE(7)
    LPS_RT_CASE(8)
    LPS_RT_CASE(9)
    LPS_RT_CASE(10)
    default: return cudaErrorNotSupported;
  }
#undef LPS_RT_CASE
}
#define LPS_RT_NZ_LIST(X) X(8) X(10) X(12) X(14) X(16) X(20) X(24) X(28) X(32)
#define LPS_RT_EXTERN(NZ) extern template cudaError_t launch_dc_rt_nz<NZ>(const DcArgs&, size_t, cudaStream_t);
LPS_RT_NZ_LIST(LPS_RT_EXTERN)
#undef LPS_RT_EXTERN

}  // namespace lps
