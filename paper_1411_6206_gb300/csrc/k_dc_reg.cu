// Data-consistency step (Algorithm 1 step 4, Sec. 3) for the 128 x 16 x-plane, with the
// Fourier transforms held in registers. One CTA per x-plane, G groups of 128 threads; each
// group takes coils grp, grp + G, ... For one coil c the plane update is
//     acc += conj(C_c) F_yz^H [M F_yz (C_c Z) - d_c]        (Z = L_k + S_k)
// with F_yz the unnormalised 2D DFT over (y, kz) (or over y per slice) scaled by
// 1/sqrt(ny nz) on each side, and M the sampled (ky, kz) lines. Per coil:
//   column phase: thread t holds the 16 samples of pixel column y = t; the length-16
//     transform along z runs in registers (dft16) and the column is stored as row kz of the
//     group's buffer;                                                      (group barrier)
//   row phase: the 8 threads of row kz (one quarter of a warp) transform it along y as
//     128 = 16 x 8: a radix-16 pass over y = j + 8r (thread j), twiddles w128^{js}, an
//     exchange through the row's own 128 shared slots, then two radix-8 passes over j
//     (thread t holds ky = s + 16q for s = t, t + 8); the residual M F(C Z) - d is formed
//     in registers from a (kz, ky) -> sampled-line map; the inverse runs the same passes
//     backwards. Only __syncwarp() separates these passes: a row never leaves its warp;
//                                                                          (group barrier)
//   column phase: inverse transform along z in registers, multiply by conj(C_c), accumulate.
// The intermediate slot of (s, j) in a row is 8 s + (j ^ (s & 7)): with a row stride of
// 136 (= 8 mod 16) complex values, every shared access of the row phase touches 16
// distinct 8-byte bank pairs per half-warp (no conflicts), as do the column accesses; the
// twiddles sit in two layouts and the line map rows 136 shorts apart for the same reason.
// The prologue forms L_k = (X_{k-1} - S_{k-1}) W (steps 1-2) and the change statistic; the
// epilogue sums the groups in a fixed order, writes X_k and the plane Gram (summed over
// 4-CTA clusters through distributed shared memory), exactly as the staged-coil kernel does.
#include "lps_internal.cuh"

#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace lps {

namespace {

constexpr int kNY = 128, kNZ = 16, kRS = 136, kGT = 128, kLMS = 136;
constexpr int kPlane = kNY * kNZ;
constexpr int kRegCluster = 4;   // x-planes per cluster (the Gram partial count nx / 4)

__device__ __forceinline__ void gsync(int bar) { asm volatile("bar.sync %0, 128;" ::"r"(bar) : "memory"); }

// ACCS: the coil terms of a group accumulate in a shared-memory column buffer of their own
// (fewer live registers) instead of registers.
template <int G, bool ACCS>
struct RegLayout {
  static constexpr size_t gbuf = (size_t)G * kNZ * kRS;   // float2
  static constexpr size_t abuf = ACCS ? gbuf : 0;
  static constexpr size_t zs = kNZ * kRS;
  static constexpr size_t bytes() {
    return (gbuf + abuf + zs + 2 * kNY + kNZ * kNZ) * sizeof(float2) + ((kNZ * kLMS * sizeof(short) + 15) & ~15) +
           64 * sizeof(float);
  }
};

// HALF: coil maps read as half-precision pairs (LPS_COILS_FP16), widened exactly to float32.
template <int G, bool FFTZ, bool ONE, bool ACCS, bool HALF, bool DH>
__global__ void __launch_bounds__(G * kGT, 1) k_dc_reg(const DcArgs a) {
  using Lay = RegLayout<G, ACCS>;
  static_assert(!(ONE && ACCS), "one coil per group needs no accumulator");
  constexpr int NTH = G * kGT;
  constexpr int EPT = kPlane / NTH;          // plane elements per thread (prologue, epilogue)
  constexpr int OUTS = kNZ * kNY / NTH;      // output slices per reprojection task
  static_assert(kPlane % NTH == 0 && kNZ % OUTS == 0, "thread count");
  const Geom& g = a.g;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* gbuf = reinterpret_cast<float2*>(smem);   // [G][kNZ][kRS]
  float2* abuf = gbuf + Lay::gbuf;                  // ACCS: [G][kNZ][kRS] coil sums
  float2* zs = abuf + Lay::abuf;                    // [kNZ][kRS]: Z, later M = X - S
  // twiddles w128^{js} (j < 8, s < 16) in two layouts, so that the index that varies across
  // the threads of a row is the contiguous one: tsj[s][j] (pass 1: j = t8) and tjs[j][s]
  // (inverse pass: s = t8 + 8h)
  float2* tsj = zs + Lay::zs;                       // [16][8]
  float2* tjs = tsj + kNY;                          // [8][16]
  float2* wsh = tjs + kNY;                          // [kNZ][kNZ]
  short* lmap = reinterpret_cast<short*>(wsh + kNZ * kNZ);   // [kNZ][kLMS]: line index or -1
  float* red = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(lmap) +
                                        ((kNZ * kLMS * sizeof(short) + 15) & ~15));

  const int tid = threadIdx.x;
  const int grp = tid / kGT, gt = tid - grp * kGT;
  const int x = blockIdx.x;
  const int nx = g.nx, ncoil = g.ncoil;
  const long long xy = (long long)nx * kNY;
  const long long xoff = (long long)x * kNY;

  for (int i = tid; i < kNY; i += NTH) {
    const int sa = i >> 3, ja = i & 7;   // tsj[sa][ja] = w^(ja sa)
    const int jb = i >> 4, sb = i & 15;  // tjs[jb][sb] = w^(jb sb)
    tsj[i] = a.tw_y[ja * sa];
    tjs[i] = a.tw_y[jb * sb];
  }
  for (int i = tid; i < kNZ * kLMS; i += NTH) lmap[i] = -1;
  // sampled-line map: (kz, ky) -> line index (lines are kz * (ny + 1) + ky in raster order);
  // the mask and its line table are set before any frame work
  const int m = a.persist->nlines;
  __syncthreads();   // the map was cleared above by other threads
  for (int l = tid; l < m; l += NTH) {
    const int p = a.lines[l];
    const int kz = p / (kNY + 1), ky = p - kz * (kNY + 1);
    lmap[kz * kLMS + ky] = (short)l;
  }
  // Iteration form with W (float32 path): this launch is released by the eigen kernel after
  // that kernel's own wait, so the previous iteration's data-consistency kernel and the sparse
  // step (joined by an event) have completed: their outputs (X_{k-1}, L_{k-1}, S_{k-1}, S_k)
  // are read before this wait, while the eigendecomposition still runs; W and the control
  // block after it.
  const bool iter_form = a.W != nullptr || a.Lpre != nullptr;
  const bool early = a.W != nullptr;
  float dz2 = 0.f, z2 = 0.f;   // ||Z_k - Z_{k-1}||^2, ||Z_{k-1}||^2 (this thread's elements)
  float2 Sk[EPT], Dz[EPT];
  float2* Mp = gbuf;                // group 0's buffer: M_{k-1} = X_{k-1} - S_{k-1}
  float2* Lsh = gbuf + kNZ * kRS;   // group 1's buffer: L_k
  auto prologue_loads = [&]() {
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int e = tid + k * NTH, z = e / kNY, y = e % kNY;
      const long long gi = (long long)z * xy + xoff + y;
      Sk[k] = a.S[gi];
      const float2 Sp = a.Sprev[gi];
      const float2 Zo = cadd(a.Lbuf[gi], Sp);
      if (a.W) Mp[z * kRS + y] = csub(a.X[gi], Sp);
      Dz[k] = csub(Sk[k], Zo);
      z2 += cabs2(Zo);
    }
  };
  if (early) prologue_loads();
  // Coil maps are set before any frame work: the column of this thread for the group's first
  // coil is loaded now; inside the loop the next coil's column is loaded one coil ahead, so
  // that its latency passes during the row phase of the current coil.
  float2 cn[kNZ];
  auto load_col = [&](int c) {
    const float2* Cc = a.coils + (long long)c * g.N + xoff + gt;
    const __half2* Ch = HALF ? a.coils_h + (long long)c * g.N + xoff + gt : nullptr;
#pragma unroll
    for (int z = 0; z < kNZ; ++z) cn[z] = HALF ? __half22float2(__ldg(Ch + z * xy)) : __ldg(Cc + z * xy);
  };
  if (grp < g.ncoil) load_col(grp);
  pdl_trigger();
  pdl_wait();   // W and the control block (without W also L, S and X) come from earlier work
  const int conv = a.ctrl ? a.ctrl->converged : 0;
  if (conv) return;   // converged earlier in this frame: nothing is written

  // ---- prologue: Z = L_k + S_k of the plane into zs -------------------------------------
  if (iter_form) {
    if (!early) prologue_loads();
    if (a.W) {
      for (int i = tid; i < kNZ * kNZ; i += NTH) wsh[i] = a.W[i];
      __syncthreads();
      // one pixel column y and OUTS output slices per task
      const int y = tid % kNY, zb = (tid / kNY) * OUTS;
      float2 o[OUTS];
#pragma unroll
      for (int j = 0; j < OUTS; ++j) o[j] = make_float2(0.f, 0.f);
#pragma unroll 4
      for (int i = 0; i < kNZ; ++i) {
        const float2 mv = Mp[i * kRS + y];
#pragma unroll
        for (int j = 0; j < OUTS; ++j) {
          const float2 w = wsh[i * kNZ + zb + j];
          o[j].x = fmaf(mv.x, w.x, fmaf(-mv.y, w.y, o[j].x));
          o[j].y = fmaf(mv.x, w.y, fmaf(mv.y, w.x, o[j].y));
        }
      }
#pragma unroll
      for (int j = 0; j < OUTS; ++j) Lsh[(zb + j) * kRS + y] = o[j];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int e = tid + k * NTH, z = e / kNY, y = e % kNY;
      const long long gi = (long long)z * xy + xoff + y;
      const float2 Lk = a.W ? Lsh[z * kRS + y] : a.Lpre[gi];
      a.Lbuf[gi] = Lk;
      dz2 += cabs2(cadd(Lk, Dz[k]));
      zs[z * kRS + y] = cadd(Lk, Sk[k]);   // Z
    }
  } else {
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int e = tid + k * NTH, z = e / kNY, y = e % kNY;
      const long long gi = (long long)z * xy + xoff + y;
      float2 v = a.L[gi];
      if (a.S) v = cadd(v, a.S[gi]);
      zs[z * kRS + y] = v;
    }
  }
  __syncthreads();

  // ---- coil loop -------------------------------------------------------------------------
  const float sc = g.scale_yz;
  const int bar = 1 + grp;
  const int row = gt >> 3, t8 = gt & 7;
  float2* B = gbuf + grp * kNZ * kRS;
  float2* R = B + row * kRS;
  const short* lrow = lmap + row * kLMS;
  // ONE: every group takes at most one coil (ncoil <= G) and writes its coil's term straight
  // into its buffer; otherwise the terms of the group's coils accumulate in registers.
  constexpr int NACC = (ONE || ACCS) ? 1 : kNZ;
  float2 acc[NACC];
#pragma unroll
  for (int z = 0; z < NACC; ++z) acc[z] = make_float2(0.f, 0.f);
  float2* A = abuf + grp * kNZ * kRS;   // ACCS: this group's sums (thread gt owns column gt)
  if (ACCS && grp >= ncoil) {
#pragma unroll
    for (int z = 0; z < kNZ; ++z) A[z * kRS + gt] = make_float2(0.f, 0.f);
  }
  float resid = 0.f;
  float2 v[16];
  if (ONE && grp >= ncoil) {
#pragma unroll
    for (int z = 0; z < kNZ; ++z) B[z * kRS + gt] = make_float2(0.f, 0.f);
  }
  for (int c = grp; c < ncoil; c += G) {
    const float2* Cc = a.coils + (long long)c * g.N + xoff + gt;
    const __half2* Ch = HALF ? a.coils_h + (long long)c * g.N + xoff + gt : nullptr;
    auto coil = [&](int z) -> float2 { return HALF ? __half22float2(__ldg(Ch + z * xy)) : __ldg(Cc + z * xy); };
    const float2* dh = a.dhyb + ((long long)x * ncoil + c) * g.mpad;
    const __half2* dhh = DH ? a.dhyb_h + ((long long)x * ncoil + c) * g.mpad : nullptr;
    // column phase: v[z] = sc C_c Z at (z, y = gt), transform along z
    const bool first = c == grp;
#pragma unroll
    for (int z = 0; z < kNZ; ++z) v[z] = cscale(cmul(cn[z], zs[z * kRS + gt]), sc);
    if (c + G < ncoil) load_col(c + G);
    if (FFTZ) dft16(v, false);
#pragma unroll
    for (int k = 0; k < kNZ; ++k) B[k * kRS + gt] = v[k];
    gsync(bar);
    // row phase, pass 1: thread j = t8 takes y = j + 8r, radix 16 over r, twiddle w128^{js}
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = R[t8 + 8 * r];
    dft16(v, false);
#pragma unroll
    for (int s = 1; s < 16; ++s) v[s] = cmul(v[s], tsj[8 * s + t8]);
    __syncwarp();
#pragma unroll
    for (int s = 0; s < 16; ++s) R[8 * s + (t8 ^ (s & 7))] = v[s];
    __syncwarp();
    // pass 2 and its inverse, one half h at a time (s = t8 + 8h). A thread reads and later
    // writes the same 8 slots 8 s + (j ^ t8), so the halves need no synchronisation.
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int s = t8 + 8 * h;
      float2 w[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) w[j] = R[8 * s + (j ^ t8)];
      int li[8];
      float2 dv[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        li[q] = lrow[s + 16 * q];
        dv[q] = li[q] >= 0 ? (DH ? __half22float2(dhh[li[q]]) : dh[li[q]]) : make_float2(0.f, 0.f);
      }
      dft8(w, false);   // radix 8 over j: w[q] = X[ky = s + 16q]
      // residual on the sampled lines (zero elsewhere)
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        float2 r = make_float2(0.f, 0.f);
        if (li[q] >= 0) {
          r = csub(w[q], dv[q]);
          resid = fmaf(r.x, r.x, fmaf(r.y, r.y, resid));
        }
        w[q] = r;
      }
      // inverse: radix 8 over q, twiddle conj(w128^{js}), back into the same slots
      dft8(w, true);
#pragma unroll
      for (int j = 1; j < 8; ++j) w[j] = cmulc(tjs[16 * j + s], w[j]);
#pragma unroll
      for (int j = 0; j < 8; ++j) R[8 * s + (j ^ t8)] = w[j];
    }
    __syncwarp();
    // radix 16 over s for j = t8: y = j + 8r
#pragma unroll
    for (int s = 0; s < 16; ++s) v[s] = R[8 * s + (t8 ^ (s & 7))];
    dft16(v, true);
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 16; ++r) R[t8 + 8 * r] = v[r];
    gsync(bar);
    // column phase: inverse along z, conj(C_c), accumulate
#pragma unroll
    for (int k = 0; k < kNZ; ++k) v[k] = B[k * kRS + gt];
    if (FFTZ) dft16(v, true);
#pragma unroll
    for (int z = 0; z < kNZ; ++z) {
      const float2 t = cmulc(coil(z), v[z]);
      if constexpr (ONE) {
        B[z * kRS + gt] = make_float2(t.x * sc, t.y * sc);   // fmaf(t, sc, 0) rounds the same
      } else if constexpr (ACCS) {
        // the first coil's term initialises the sum (0 + t sc rounds the same)
        float2 u = first ? make_float2(0.f, 0.f) : A[z * kRS + gt];
        u.x = fmaf(t.x, sc, u.x);
        u.y = fmaf(t.y, sc, u.y);
        A[z * kRS + gt] = u;
      } else {
        acc[z].x = fmaf(t.x, sc, acc[z].x);
        acc[z].y = fmaf(t.y, sc, acc[z].y);
      }
    }
    // the next coil's column writes touch only this thread's own column: no barrier needed
  }

  // ---- epilogue: X_k = Z - sum over groups (fixed order), M = X_k - S_k, plane Gram ------
  if constexpr (!ONE && !ACCS) {
#pragma unroll
    for (int z = 0; z < kNZ; ++z) B[z * kRS + gt] = acc[z];
  }
  __syncthreads();
  const float2* sums = ACCS ? abuf : gbuf;
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int e = tid + k * NTH, z = e / kNY, y = e % kNY;
    const long long gi = (long long)z * xy + xoff + y;
    float2 s = sums[z * kRS + y];
#pragma unroll
    for (int q = 1; q < G; ++q) s = cadd(s, sums[q * kNZ * kRS + z * kRS + y]);
    const float2 Zv = zs[z * kRS + y];
    const float2 Xv = csub(Zv, s);
    if (a.recon) a.recon[gi] = Zv;
    a.X[gi] = Xv;
    zs[z * kRS + y] = a.S ? csub(Xv, a.S[gi]) : Xv;   // same element, same thread
  }
  __syncthreads();
  if (a.gram_part) {
    // plane Gram: one warp per column pair (i <= j), lanes across y
    constexpr int NPAIR = kNZ * (kNZ + 1) / 2;
    constexpr int NW = NTH / 32;
    const int w = tid >> 5, lane = tid & 31;
    float2* gsm = gbuf;   // group 0's buffer is free again
    for (int pr = w; pr < NPAIR; pr += NW) {
      int i = 0, rem = pr;
      while (rem >= kNZ - i) {
        rem -= kNZ - i;
        ++i;
      }
      const int j = i + rem;
      const float2* ri = zs + i * kRS;
      const float2* rj = zs + j * kRS;
      float sr = 0.f, si = 0.f;
#pragma unroll
      for (int y = lane; y < kNY; y += 32) {
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
        gsm[i * kNZ + j] = make_float2(sr, si);
        if (i != j) gsm[j * kNZ + i] = make_float2(sr, -si);
      }
    }
    // cluster sum in a fixed rank order
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();
    const int rank = (int)cl.block_rank();
    float2* gp = a.gram_part + (long long)(x / kRegCluster) * kNZ * kNZ;
    for (int e = rank + kRegCluster * tid; e < kNZ * kNZ; e += kRegCluster * NTH) {
      float2 acc2 = make_float2(0.f, 0.f);
#pragma unroll
      for (int r = 0; r < kRegCluster; ++r) acc2 = cadd(acc2, cl.map_shared_rank(gsm, r)[e]);
      gp[e] = acc2;
    }
    cl.sync();   // no CTA leaves while another still reads its shared memory
  }
  if (a.dc_part) {
    const float r2 = block_sum(resid, red);
    const float d2 = block_sum(dz2, red);
    const float o2 = block_sum(z2, red);
    if (tid == 0) reinterpret_cast<float4*>(a.dc_part)[x] = make_float4(r2, d2, o2, 0.f);
  }
}

template <int G, bool FFTZ, bool ONE, bool ACCS, bool HALF, bool DH = false>
cudaError_t launch_reg(const DcArgs& a, cudaStream_t st) {
  constexpr size_t smem = RegLayout<G, ACCS>::bytes();
  static_assert(smem <= 227 * 1024, "shared memory");
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e =
        cudaFuncSetAttribute(k_dc_reg<G, FFTZ, ONE, ACCS, HALF, DH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(a.g.nx);
  cfg.blockDim = dim3(G * kGT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = kRegCluster;
  attr[1].val.clusterDim.y = 1;
  attr[1].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_dc_reg<G, FFTZ, ONE, ACCS, HALF, DH>, a);
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace

// The register-transform kernel covers the update form (steps 1-4 of an iteration, or
// step 4 alone) of the 128 x 16 plane; the caller falls back to the other kernels on
// cudaErrorNotSupported. It writes the same Gram partial count as the staged-coil kernel
// (nx / 4, one per 4-plane cluster).
bool dc_reg_applies(const Geom& g) {
  return !g.dc_generic && g.cs == 1 && g.ny == kNY && g.nz == kNZ && g.nx % kRegCluster == 0 && g.dc_reg_groups > 0;
}

cudaError_t launch_dc_reg(const DcArgs& a, cudaStream_t st) {
  if (!dc_reg_applies(a.g)) return cudaErrorNotSupported;
  const bool fz = a.g.fft_z != 0;
  // dc_reg_groups: 4 or 8 coil groups; 104: four groups with their coil sums in shared memory
  // (used when there are more coils than groups). Half-precision coil maps: four groups.
  const bool accs = a.g.dc_reg_groups > 100;
  // half-precision samples (LPS_DATA_FP16) are read as half pairs by the four-group variants
  // with one coil per group or the coil sums in shared memory (the defaults); the others read
  // the rounded float32 copy (the same values)
  if (a.dhyb_h && a.g.dc_reg_groups % 100 == 4 && (a.g.ncoil <= 4 || accs)) {
    const bool one = a.g.ncoil <= 4;
    if (a.coils_h) {
      if (one) return fz ? launch_reg<4, true, true, false, true, true>(a, st) : launch_reg<4, false, true, false, true, true>(a, st);
      return fz ? launch_reg<4, true, false, true, true, true>(a, st) : launch_reg<4, false, false, true, true, true>(a, st);
    }
    if (one) return fz ? launch_reg<4, true, true, false, false, true>(a, st) : launch_reg<4, false, true, false, false, true>(a, st);
    return fz ? launch_reg<4, true, false, true, false, true>(a, st) : launch_reg<4, false, false, true, false, true>(a, st);
  }
  if (a.coils_h && a.g.dc_reg_groups % 100 == 4) {
    if (a.g.ncoil <= 4) return fz ? launch_reg<4, true, true, false, true>(a, st) : launch_reg<4, false, true, false, true>(a, st);
    if (accs) return fz ? launch_reg<4, true, false, true, true>(a, st) : launch_reg<4, false, false, true, true>(a, st);
    return fz ? launch_reg<4, true, false, false, true>(a, st) : launch_reg<4, false, false, false, true>(a, st);
  }
  switch (a.g.dc_reg_groups % 100) {
    case 4:
      if (a.g.ncoil <= 4) return fz ? launch_reg<4, true, true, false, false>(a, st) : launch_reg<4, false, true, false, false>(a, st);
      if (accs) return fz ? launch_reg<4, true, false, true, false>(a, st) : launch_reg<4, false, false, true, false>(a, st);
      return fz ? launch_reg<4, true, false, false, false>(a, st) : launch_reg<4, false, false, false, false>(a, st);
    case 8:
      if (a.g.ncoil <= 8) return fz ? launch_reg<8, true, true, false, false>(a, st) : launch_reg<8, false, true, false, false>(a, st);
      return fz ? launch_reg<8, true, false, false, false>(a, st) : launch_reg<8, false, false, false, false>(a, st);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace lps
