// Data-consistency step (Algorithm 1 step 4, Sec. 3) and acquisition operator (Sec. 2) for
// plane sizes fixed at compile time. Same arithmetic as k_dc (hybrid-space formulation,
// one CTA per x-plane), specialised so that every Stockham pass is unrolled with constant
// strides and radices:
//   - NCG coil groups of NT threads run concurrently, each on its own coils, shared-memory
//     buffers, TMA double buffer and named barrier; their coil sums are added in a fixed order
//     at the end (deterministic);
//   - in the iteration form the prologue completes steps (1)-(2) for the plane,
//     L_k = (X_{k-1} - S_{k-1}) W, and the change statistic ||Z_k - Z_{k-1}||;
//   - the plane Gram epilogue assigns one warp per (i <= j) column pair, lanes across y.
#include "lps_internal.cuh"

#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace lps {

// CTAs (x-planes) per cluster: their plane Grams are summed through distributed shared
// memory, so the eigen kernel reads nx / kGramCluster partials instead of nx.
constexpr int kGramCluster = 4;

__host__ __device__ constexpr int ct_radix(int rem) {
  return (rem % 16 == 0 && rem != 32) ? 16
         : (rem % 8 == 0)             ? 8
         : (rem % 4 == 0)             ? 4
         : (rem % 2 == 0)             ? 2
         : (rem % 3 == 0)             ? 3
         : (rem % 5 == 0)             ? 5
         : (rem % 7 == 0)             ? 7
                                      : rem;
}

__device__ __forceinline__ void group_sync(int bar, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nthreads) : "memory");
}

// OR of `v` over the `nthreads` threads of named barrier `bar` (also a barrier).
__device__ __forceinline__ bool group_or(int bar, int nthreads, bool v) {
  unsigned r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((unsigned)v), "r"(bar), "r"(nthreads)
      : "memory");
  return r != 0;
}

template <int N, int NB, int ES, int BS, int NS, int R, int NT, bool INV>
__device__ __forceinline__ void ct_pass(const float2* __restrict__ in, float2* __restrict__ out,
                                        const float2* __restrict__ tw, int gtid) {
  constexpr int NBF = N / R;
  constexpr int TOTAL = NB * NBF;
  constexpr int TWS = N / (NS * R);
  constexpr int ITER = (TOTAL + NT - 1) / NT;
#pragma unroll
  for (int it = 0; it < ITER; ++it) {
    const int t = gtid + it * NT;
    if ((TOTAL % NT) != 0 && t >= TOTAL) break;
    const int b = t % NB;
    const int j = t / NB;
    const int k = j % NS;
    float2 v[R];
    const float2* src = in + b * BS + j * ES;
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[r * NBF * ES];
    if constexpr (NS > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        float2 w = tw[r * k * TWS];
        if (INV) w.y = -w.y;
        v[r] = cmul(v[r], w);
      }
    }
    dft_reg<R>(v, INV, tw, N);
    float2* dst = out + b * BS + ((j / NS) * NS * R + k) * ES;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[r * NS * ES] = v[r];
  }
}

// All passes of a length-N transform over NB batches; result pointer returned.
template <int N, int NB, int ES, int BS, int NS, int NT, bool INV>
__device__ __forceinline__ float2* ct_fft(float2* src, float2* dst, const float2* tw, int gtid, int bar) {
  if constexpr (NS >= N) {
    return src;
  } else {
    constexpr int R = ct_radix(N / NS);
    ct_pass<N, NB, ES, BS, NS, R, NT, INV>(src, dst, tw, gtid);
    group_sync(bar, NT);
    return ct_fft<N, NB, ES, BS, NS * R, NT, INV>(dst, src, tw, gtid, bar);
  }
}

template <int NY, int NZ, int NCG, int NT>
struct DcFixedLayout {
  static constexpr int NYP = NY + 1;
  static constexpr int PLANE = NY * NZ;
  static constexpr int PLANEP = (NZ * NYP + 1) & ~1;
  static constexpr int EPT = (PLANE + NT - 1) / NT;
  static constexpr int GROUP = 2 * PLANEP + 2 * PLANE;   // complex elements per coil group
  static constexpr size_t bytes() {
    return (size_t)(NCG * GROUP + NY + NZ + ((NY + NZ) & 1)) * sizeof(float2) + 2 * NCG * sizeof(uint64_t) +
           64 * sizeof(float) + (size_t)NZ * NZ * sizeof(float2);   // ..., reduction scratch, W
  }
};

template <int NY, int NZ, int NCG, int NT, int MODE>
__global__ void __launch_bounds__(NCG* NT, 1) k_dc_fixed(const DcArgs a) {
  using Lay = DcFixedLayout<NY, NZ, NCG, NT>;
  constexpr int NYP = Lay::NYP, PLANE = Lay::PLANE, PLANEP = Lay::PLANEP, EPT = Lay::EPT;
  constexpr int NTH = NCG * NT;
  const Geom& g = a.g;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* base = reinterpret_cast<float2*>(smem);
  float2* twy = base + NCG * Lay::GROUP;
  float2* twz = twy + NY;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(twz + NZ + ((NY + NZ) & 1));
  float* red = reinterpret_cast<float*>(mbar + 2 * NCG);
  float2* wsh = reinterpret_cast<float2*>(red + 64);   // [NZ][NZ] W of the iteration form

  const int tid = threadIdx.x;
  const int grp = tid / NT, gtid = tid - grp * NT;
  const int bar = 1 + grp;
  float2* bufA = base + grp * Lay::GROUP;
  float2* bufB = bufA + PLANEP;
  float2* coilS0 = bufB + PLANEP;
  float2* coilS1 = coilS0 + PLANE;
  uint64_t* gbar = mbar + 2 * grp;
  const int x = blockIdx.x;
  const int nx = g.nx, ncoil = g.ncoil;
  const long long xy = (long long)nx * NY;
  int* errp = a.ctrl ? &a.ctrl->err : nullptr;
  constexpr unsigned kRowBytes = NY * sizeof(float2);
  auto issue = [&](int c, float2* slot, uint64_t* b) {
    mbar_arrive_expect_tx(b, kRowBytes * NZ);
    const float2* src = a.coils + (long long)c * g.N + (long long)x * NY;
#pragma unroll 4
    for (int z = 0; z < NZ; ++z) bulk_g2s(slot + z * NY, src + z * xy, kRowBytes, b);
  };
  // The first two coil planes of each group are requested before anything else; the
  // control flag and the other global inputs are loaded while they are in flight.
  unsigned inflight = 0;   // slots with a copy in flight (thread gtid == 0 of each group)
  unsigned phase = 0;      // parity of the next phase to wait for, per slot
  if (gtid == 0) {
    mbar_init(&gbar[0], 1);
    mbar_init(&gbar[1], 1);
    fence_mbar_init();
    if (grp < ncoil) {
      issue(grp, coilS0, &gbar[0]);
      inflight |= 1u;
    }
    if (grp + NCG < ncoil) {
      issue(grp + NCG, coilS1, &gbar[1]);
      inflight |= 2u;
    }
  }
  for (int i = tid; i < NY; i += NTH) twy[i] = a.tw_y[i];
  for (int i = tid; i < NZ; i += NTH) twz[i] = a.tw_z[i];
  pdl_trigger();
  pdl_wait();   // L, S, the control block and the line count come from earlier work
  const int conv = a.ctrl ? a.ctrl->converged : 0;
  const int m = a.persist->nlines;

  float2 Zr[EPT], acc[EPT];
  float dz2 = 0.f, z2 = 0.f;   // ||Z_k - Z_{k-1}||^2 and ||Z_{k-1}||^2 (group 0's elements)
  // Iteration form (Algorithm 1) or operator form (Z = L + S given); nothing is read once the
  // frame has converged (the iteration form leaves a.L null).
  const bool iter_form = MODE == kDcUpdate && (a.W != nullptr || a.Lpre != nullptr);
  if (conv) {
#pragma unroll
    for (int k = 0; k < EPT; ++k) Zr[k] = acc[k] = make_float2(0.f, 0.f);
  } else if (iter_form) {
    // Steps (1)-(2) completed here: L_k = (X_{k-1} - S_{k-1}) W, column by column of the
    // Casorati matrix (the x-plane holds every slice of its pixels), or the precomputed L_k.
    float2* Mp = base;            // group 0's first buffer: M_{k-1} as [z][NYP]
    float2* Lsh = base + PLANEP;  // group 0's second buffer: L_k as [z][NYP]
    // Every per-element global load is issued here, before the product, so that their
    // latencies overlap: S_k for each group; in group 0 also X_{k-1}, S_{k-1} and L_{k-1},
    // giving M_{k-1} (into shared memory) and S_k - Z_{k-1} (kept for the change statistic).
    float2 Dz[EPT];
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int e = gtid + k * NT;
      Zr[k] = Dz[k] = make_float2(0.f, 0.f);
      acc[k] = make_float2(0.f, 0.f);
      if (PLANE % NT == 0 || e < PLANE) {
        const int z = e / NY, y = e % NY;
        const long long gi = (long long)z * xy + (long long)x * NY + y;
        Zr[k] = a.S[gi];
        if (grp == 0) {
          const float2 Sp = a.Sprev[gi];
          const float2 Zo = cadd(a.Lbuf[gi], Sp);
          if (a.W) Mp[z * NYP + y] = csub(a.X[gi], Sp);
          Dz[k] = csub(Zr[k], Zo);
          z2 += cabs2(Zo);
        }
      }
    }
    if (a.W) {
      for (int i = tid; i < NZ * NZ; i += NTH) wsh[i] = a.W[i];
      __syncthreads();
      // one pixel column y and 8 output slices per task: M[i][y] read once per 8 products,
      // W rows broadcast across the warp
      for (int task = tid; task < NY * (NZ / 8); task += NTH) {
        const int y = task % NY, zb = (task / NY) * 8;
        float2 o[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) o[j] = make_float2(0.f, 0.f);
#pragma unroll 4
        for (int i = 0; i < NZ; ++i) {
          const float2 mv = Mp[i * NYP + y];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const float2 w = wsh[i * NZ + zb + j];
            o[j].x = fmaf(mv.x, w.x, fmaf(-mv.y, w.y, o[j].x));
            o[j].y = fmaf(mv.x, w.y, fmaf(mv.y, w.x, o[j].y));
          }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) Lsh[(zb + j) * NYP + y] = o[j];
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int e = gtid + k * NT;
      if (PLANE % NT == 0 || e < PLANE) {
        const int z = e / NY, y = e % NY;
        const long long gi = (long long)z * xy + (long long)x * NY + y;
        const float2 Lk = a.W ? Lsh[z * NYP + y] : a.Lpre[gi];
        Zr[k] = cadd(Lk, Zr[k]);
        if (grp == 0) {
          a.Lbuf[gi] = Lk;
          dz2 += cabs2(cadd(Lk, Dz[k]));
        }
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int e = gtid + k * NT;
      acc[k] = make_float2(0.f, 0.f);
      Zr[k] = make_float2(0.f, 0.f);
      if ((PLANE % NT == 0 || e < PLANE) && MODE != kDcAdjoint) {
        const int z = e / NY, y = e % NY;
        const long long gi = (long long)z * xy + (long long)x * NY + y;
        float2 v = a.L[gi];
        if (MODE == kDcUpdate && a.S) v = cadd(v, a.S[gi]);
        Zr[k] = v;
      }
    }
  }
  __syncthreads();
  if (conv) {
    // converged earlier in this frame: let the copies land, then leave
    if (gtid == 0)
      for (int s = 0; s < 2; ++s)
        if (inflight & (1u << s)) mbar_wait_bounded(&gbar[s], 0u, nullptr);
    return;
  }

  const float sc = g.scale_yz;
  float resid = 0.f;
  int u = 0;
  bool bad_any = false;
  for (int c = grp; c < ncoil; c += NCG, ++u) {
    const int s = u & 1;
    float2* coil = s ? coilS1 : coilS0;
    const bool bad = !mbar_wait_bounded(&gbar[s], (phase >> s) & 1u, errp);
    if (group_or(bar, NT, bad)) {
      bad_any = true;
      break;
    }
    phase ^= 1u << s;
    if (gtid == 0) inflight &= ~(1u << s);
    float2* src = bufA;
    float2* dst = bufB;
    const float2* dh = a.dhyb + ((long long)x * ncoil + c) * g.mpad;
    if (MODE != kDcAdjoint) {
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int e = gtid + k * NT;
        if (PLANE % NT == 0 || e < PLANE) src[(e / NY) * NYP + e % NY] = cscale(cmul(coil[e], Zr[k]), sc);
      }
      group_sync(bar, NT);
      src = ct_fft<NY, NZ, 1, NYP, 1, NT, false>(src, dst, twy, gtid, bar);
      dst = (src == bufA) ? bufB : bufA;
      if (g.fft_z) {
        src = ct_fft<NZ, NY, NYP, 1, 1, NT, false>(src, dst, twz, gtid, bar);
        dst = (src == bufA) ? bufB : bufA;
      }
      if (MODE == kDcForward) {
        float2* ho = a.hyb_out + ((long long)x * ncoil + c) * g.mpad;
        for (int l = gtid; l < m; l += NT) ho[l] = src[a.lines[l]];
        group_sync(bar, NT);
        if (gtid == 0 && c + 2 * NCG < ncoil) {
          fence_proxy_async();
          issue(c + 2 * NCG, coil, &gbar[s]);
          inflight |= 1u << s;
        }
        continue;
      }
    }
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int e = gtid + k * NT;
      if (PLANE % NT == 0 || e < PLANE) dst[(e / NY) * NYP + e % NY] = make_float2(0.f, 0.f);
    }
    group_sync(bar, NT);
    for (int l = gtid; l < m; l += NT) {
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
    group_sync(bar, NT);
    src = dst;
    dst = (src == bufA) ? bufB : bufA;
    if (g.fft_z) {
      src = ct_fft<NZ, NY, NYP, 1, 1, NT, true>(src, dst, twz, gtid, bar);
      dst = (src == bufA) ? bufB : bufA;
    }
    src = ct_fft<NY, NZ, 1, NYP, 1, NT, true>(src, dst, twy, gtid, bar);
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int e = gtid + k * NT;
      if (PLANE % NT == 0 || e < PLANE) {
        const float2 v = cmulc(coil[e], src[(e / NY) * NYP + e % NY]);
        acc[k].x = fmaf(v.x, sc, acc[k].x);
        acc[k].y = fmaf(v.y, sc, acc[k].y);
      }
    }
    group_sync(bar, NT);
    if (gtid == 0 && c + 2 * NCG < ncoil) {
      fence_proxy_async();
      issue(c + 2 * NCG, coil, &gbar[s]);
      inflight |= 1u << s;
    }
  }
  // agree on failure across the whole CTA (named-barrier groups finished their loops)
  if (__syncthreads_or(bad_any)) {
    if (gtid == 0) {
      for (int s = 0; s < 2; ++s)
        if (inflight & (1u << s)) mbar_wait_bounded(&gbar[s], (phase >> s) & 1u, nullptr);
    }
    return;
  }
  if (MODE == kDcForward) return;

  // Sum the coil groups in a fixed order: groups >= 1 park their sums in their bufA.
  if (NCG > 1 && grp > 0) {
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int e = gtid + k * NT;
      if (PLANE % NT == 0 || e < PLANE) bufA[e] = acc[k];
    }
  }
  __syncthreads();
  float2* M = base;   // group 0's bufA holds M = X - S for the Gram
  if (grp == 0) {
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int e = gtid + k * NT;
      if (PLANE % NT == 0 || e < PLANE) {
        float2 sacc = acc[k];
        for (int q = 1; q < NCG; ++q) sacc = cadd(sacc, base[q * Lay::GROUP + e]);
        const int z = e / NY, y = e % NY;
        const long long gi = (long long)z * xy + (long long)x * NY + y;
        float2 Xv, Mv;
        if (MODE == kDcUpdate) {
          Xv = csub(Zr[k], sacc);
          if (a.recon) a.recon[gi] = Zr[k];
          Mv = a.S ? csub(Xv, a.S[gi]) : Xv;
        } else {
          Xv = sacc;
          Mv = Xv;
          if (a.L_out) a.L_out[gi] = Xv;
          if (a.S_out) a.S_out[gi] = make_float2(0.f, 0.f);
        }
        a.X[gi] = Xv;
        M[z * NYP + y] = Mv;
      }
    }
  }
  __syncthreads();
  if (a.gram_part) {
    // Plane Gram into shared memory: one warp per column pair (i <= j), lanes across y.
    constexpr int NPAIR = NZ * (NZ + 1) / 2;
    constexpr int NW = NTH / 32;
    const int w = tid >> 5, lane = tid & 31;
    float2* gsm = base + PLANEP;   // group 0's second FFT buffer is free now
    for (int pr = w; pr < NPAIR; pr += NW) {
      int i = 0, rem = pr;
      while (rem >= NZ - i) {
        rem -= NZ - i;
        ++i;
      }
      const int j = i + rem;
      const float2* ri = M + i * NYP;
      const float2* rj = M + j * NYP;
      float sr = 0.f, si = 0.f;
#pragma unroll
      for (int y = lane; y < NY; y += 32) {
        const float2 p = ri[y], q = rj[y];
        sr = fmaf(p.x, q.x, fmaf(p.y, q.y, sr));
        si = fmaf(p.x, q.y, fmaf(-p.y, q.x, si));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        si += __shfl_xor_sync(0xffffffffu, si, o);
      }
      if (lane == 0) {
        gsm[i * NZ + j] = make_float2(sr, si);
        if (i != j) gsm[j * NZ + i] = make_float2(sr, -si);
      }
    }
    // Cluster sum in a fixed rank order: CTA `rank` adds entries e = rank (mod cluster) over
    // the cluster's planes and writes the cluster's partial.
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();
    const int rank = (int)cl.block_rank();
    float2* gp = a.gram_part + (long long)(x / kGramCluster) * NZ * NZ;
    for (int e = rank + kGramCluster * tid; e < NZ * NZ; e += kGramCluster * NTH) {
      float2 acc2 = make_float2(0.f, 0.f);
#pragma unroll
      for (int r = 0; r < kGramCluster; ++r) acc2 = cadd(acc2, cl.map_shared_rank(gsm, r)[e]);
      gp[e] = acc2;
    }
    cl.sync();   // no CTA leaves while another still reads its shared memory
  }
  if (MODE == kDcUpdate && a.dc_part) {
    const float r2 = block_sum(resid, red);
    const float d2 = block_sum(dz2, red);
    const float o2 = block_sum(z2, red);
    if (tid == 0) reinterpret_cast<float4*>(a.dc_part)[x] = make_float4(r2, d2, o2, 0.f);
  }
}

template <int NY, int NZ, int NCG, int NT, int MODE>
static cudaError_t launch_fixed(const DcArgs& a, cudaStream_t st) {
  using Lay = DcFixedLayout<NY, NZ, NCG, NT>;
  constexpr size_t smem = Lay::bytes();
  static_assert(smem <= 227 * 1024, "plane does not fit shared memory");
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_dc_fixed<NY, NZ, NCG, NT, MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(a.g.nx);
  cfg.blockDim = dim3(NCG * NT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = kGramCluster;
  attr[1].val.clusterDim.y = 1;
  attr[1].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_dc_fixed<NY, NZ, NCG, NT, MODE>, a);
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <int NY, int NZ, int NCG, int NT>
static cudaError_t launch_fixed_mode(const DcArgs& a, int mode, cudaStream_t st) {
  switch (mode) {
    case kDcUpdate: return launch_fixed<NY, NZ, NCG, NT, kDcUpdate>(a, st);
    case kDcAdjoint: return launch_fixed<NY, NZ, NCG, NT, kDcAdjoint>(a, st);
    default: return launch_fixed<NY, NZ, NCG, NT, kDcForward>(a, st);
  }
}

static bool has_fixed(const Geom& g) {
  if (g.dc_generic || g.cs != 1 || g.nx % kGramCluster != 0) return false;   // whole clusters (nx % 8 == 0 anyway)
  return (g.ny == 128 && g.nz == 16) || (g.ny == 192 && g.nz == 32) || (g.ny == 32 && g.nz == 8);
}

// Number of Gram partials the data-consistency step leaves for the eigen kernel.
int dc_gram_parts(const Geom& g) { return has_fixed(g) ? g.nx / kGramCluster : g.nx; }

bool dc_has_fixed(const Geom& g) { return has_fixed(g); }

// Returns cudaErrorNotSupported when no specialisation matches (the caller falls back to the
// runtime-sized kernel).
cudaError_t launch_dc_fixed(const DcArgs& a, int mode, cudaStream_t st) {
  const Geom& g = a.g;
  if (!has_fixed(g)) return cudaErrorNotSupported;
  if (g.ny == 128 && g.nz == 16) return launch_fixed_mode<128, 16, 2, 256>(a, mode, st);
  if (g.ny == 192 && g.nz == 32) return launch_fixed_mode<192, 32, 1, 512>(a, mode, st);
  if (g.ny == 32 && g.nz == 8) return launch_fixed_mode<32, 8, 1, 256>(a, mode, st);
  return cudaErrorNotSupported;
}

}  // namespace lps
