// Steps (1) and (2) of Algorithm 1 (Sec. 3) on the small side of the Casorati matrix.
//
// The singular values and right singular vectors of M = X - S (N_r x nc, N_r >> nc) are
// those of its Gram matrix G = M^H M = V diag(sigma^2) V^H. One CTA:
//   1. records the statistics of the previous iteration (residual, nuclear norm, l1 off the
//      prior support, relative change; the host forms the objective from them) and applies
//      the stopping rule (Sec. 3: stop when the relative change of the solution falls below
//      the tolerance);
//   2. sums the Gram partials of the data-consistency step in float32 (one or two
//      interleaved chunk sums per entry, combined in a fixed order);
//   3. diagonalises G by cyclic two-sided Jacobi rotations in round-robin order, starting
//      from A = V_prev^H G V_prev with the previous eigenvectors; each step computes the
//      nc/2 disjoint rotations, then updates every element of A (J^H A J) and every column
//      pair of V (V J) in parallel (float64 mode: refined afterwards by k_ritz64_a/b);
//   4. sigma = sqrt(lambda), step (1) sigma' = max(sigma - lambda_L, 0), step (2)
//      sigma'' = sigma' - lambda_p (sigma' - sigma_prev) (matched by rank), rank guard
//      sigma''_i = 0 where sigma_i <= tau sigma_1;
//   5. writes W = V diag(sigma''/sigma) V^H so that L = M W = U diag(sigma'') V^H.
// At the first iteration it also fixes lambda_L = rel_L sigma_1(X_0) and
// lambda_S = rel_S max|T(X_0)|.
#include "lps_internal.cuh"

namespace lps {

constexpr int kEigThreads = 512;
constexpr int kLd = kMaxNc + 1;   // leading dimension of the shared matrices

__device__ __forceinline__ float2 mkc(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ double2 mkc(double x, double y) { return make_double2(x, y); }
template <typename C>
__device__ __forceinline__ C add_(C a, C b) { return mkc(a.x + b.x, a.y + b.y); }
template <typename C>
__device__ __forceinline__ C sub_(C a, C b) { return mkc(a.x - b.x, a.y - b.y); }
template <typename C>
__device__ __forceinline__ C mul_(C a, C b) { return mkc(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename C>
__device__ __forceinline__ C mulc_(C a, C b) { return mkc(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }  // conj(a) b
template <typename C, typename R>
__device__ __forceinline__ C scl_(C a, R s) { return mkc(a.x * s, a.y * s); }
template <typename C>
__device__ __forceinline__ C conj_(C a) { return mkc(a.x, -a.y); }

// Approximate reciprocal square root with subnormals flushed to zero (PTX rsqrt.approx.ftz):
// the rotation parameters need neither the subnormal range nor the extra instructions that
// preserve it.
__device__ __forceinline__ float rsqrt_ftz(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Rotation of a pair (p, q): J = [[c, se], [-conj(se), c]] with se = s a_pq/|a_pq| and
// t = tan(theta) from tau = (a_qq - a_pp)/(2|a_pq|), t = sign(tau)/(|tau| + sqrt(1 + tau^2))
// (the smaller root). Packed as {c, se.x, se.y, t|a_pq|}; t|a_pq| = 0 means no rotation.
// A pair is left alone when |a_pq| <= max(eps max(|a_pp|, |a_qq|), floor): below that a
// rotation moves the eigenvalues by O(eps^2 a) and the vectors by O(eps), the rounding level
// of the arithmetic; `floor` (about one unit in the last place of the trace) stops
// rotations of pairs of near-zero eigenvalues that only exchange rounding noise.
__device__ __forceinline__ float4 rot_params(const float2* A, int p, int q, float eps, float floor_) {
  const float app = A[p * kLd + p].x, aqq = A[q * kLd + q].x;
  const float2 apq = A[p * kLd + q];
  const float g2 = apq.x * apq.x + apq.y * apq.y;
  const float lim = fmaxf(eps * fmaxf(fabsf(app), fabsf(aqq)), floor_);
  // Computed for every pair and selected at the end (no divergent branch in the Jacobi
  // step), from r = sqrt(d^2 + 4|a_pq|^2), d = a_qq - a_pp, through two dependent approximate
  // reciprocal square roots: with rq = 1/r, cos^2(theta) = x = (1 + |d| rq)/2, so
  // c = x / sqrt(x), s e^{i arg a_pq} = sign(d) rq / sqrt(x) a_pq (|s| = |a_pq| / (r c)) and
  // t|a_pq| = sign(d) |a_pq|^2 rq / x (t = tan(theta), the smaller root). In exact arithmetic
  // c^2 + |s|^2 = x + |a_pq|^2 rq^2 / x = 1; in float32 it holds to a few units in the last
  // place, as does the annihilation of a_pq; a residue left in a_pq is removed by the next
  // sweep.
  float4 r;
  const bool rot = g2 > lim * lim;
  const float d = aqq - app;
  const float q2 = fmaf(4.0f, g2, d * d);
  const float rq = rsqrt_ftz(rot ? q2 : 1.0f);   // q2 itself whenever the pair rotates
  const float x = fmaf(0.5f * fabsf(d), rq, 0.5f);
  const float ix = rsqrt_ftz(x);
  const float c = x * ix;
  const float fs = copysignf(rq * ix, d);
  r.x = rot ? c : 1.f;
  r.y = rot ? fs * apq.x : 0.f;
  r.z = rot ? fs * apq.y : 0.f;
  r.w = rot ? fs * ix * g2 : 0.f;
  return r;
}

// Position of an index after one step of the circle schedule. The matrix is kept in
// "position" order: step s rotates the pairs of positions (2k, 2k+1), then every element
// moves to its next position, so that the next step again pairs (2k, 2k+1). Position 0 is
// fixed; the others move along the ring 1 -> 2 -> 4 -> ... -> np-2 -> np-1 -> np-3 -> ... -> 3
// -> 1 of length np-1 (odd). Two ring elements share a pair when they sit symmetrically
// about position 1 of the ring, and each unordered pair has one such step per np-1 steps,
// so np-1 steps (one sweep) meet every pair once and bring every index back to its own
// position.
__device__ __forceinline__ int next_pos(int p, int np) {
  if (np == 2 || p == 0) return p;
  if (p == 1) return 2;
  if ((p & 1) == 0) return p == np - 2 ? np - 1 : p + 2;
  return p - 2;
}

// Cyclic Jacobi on the Hermitian n x n matrix in A (zero-padded to even np); the
// eigenvectors are accumulated into V (V <- V J per rotation). An and Vn are the second
// buffers of the position permutation; on return A and V point at the results (index
// order). Each thread keeps one task over all steps, since the tasks address positions:
// either a block (k1 <= k2) of the 2 x 2 blocks of A, which it rotates on both sides with
// the rotations of pairs k1 and k2 and writes (with its mirror) at the moved positions, or
// two rows of V at pair k2. The three kinds of task (off-diagonal blocks, diagonal blocks,
// V rows) start on warp boundaries, so that no warp splits between their code paths. Every
// thread computes the rotations it needs itself from the diagonal blocks, so one barrier per
// step suffices. Returns the sweeps done.
// Threads that hold a task of the Jacobi step below (whole warps): off-diagonal blocks from
// thread 0, diagonal blocks and V row pairs each from the next warp boundary.
__host__ __device__ __forceinline__ int jacobi_threads(int n) {
  const int np = n + (n & 1), nh = np >> 1;
  const int noff = nh * (nh - 1) / 2;
  const int dbase = ((noff + 31) >> 5) << 5;
  const int vbase = ((dbase + nh + 31) >> 5) << 5;
  return ((vbase + nh * nh + 31) >> 5) << 5;
}

__device__ __forceinline__ void jsync(int nthr) { asm volatile("bar.sync 1, %0;" ::"r"(nthr) : "memory"); }

// Called by threads 0 .. jacobi_threads(n) - 1 only (named barrier 1): the other warps of the
// CTA have no task and wait at the CTA barrier that follows.
template <int NCT>
__device__ int jacobi(float2*& A, float2*& An, float2*& V, float2*& Vn, int n_rt, float eps, float floor_,
                      int max_sweeps, float start, int* flags) {
  const int n = NCT ? NCT : n_rt;
  const int nthr = jacobi_threads(n);
  using C = float2;
  using C4 = float4;
  using R = float;
  const int np = n + (n & 1);
  const int nh = np >> 1;
  const int noff = nh * (nh - 1) / 2;           // off-diagonal blocks k1 < k2 from thread 0
  const int dbase = ((noff + 31) >> 5) << 5;      // diagonal blocks
  const int vbase = ((dbase + nh + 31) >> 5) << 5;   // V row pairs (at most 416 threads: n <= 32)
  const int tid = threadIdx.x;
  int role = 0, k1 = 0, k2 = 0, r0 = 0;
  if (tid < noff) {
    role = 1;
    int t = tid;
    while (t >= nh - 1 - k1) {
      t -= nh - 1 - k1;
      ++k1;
    }
    k2 = k1 + 1 + t;
  } else if (tid >= dbase && tid < dbase + nh) {
    role = 1;
    k1 = k2 = tid - dbase;
  } else if (tid >= vbase && tid < vbase + nh * nh) {
    role = 2;
    const int t = tid - vbase;
    k2 = t % nh;
    r0 = 2 * (t / nh);
  }
  const int p1 = 2 * k1, q1 = p1 + 1, p2 = 2 * k2, q2 = p2 + 1;
  const int np1 = next_pos(p1, np), nq1 = next_pos(q1, np);
  const int np2 = next_pos(p2, np), nq2 = next_pos(q2, np);
  int sweep = 0;
  for (;;) {
    // converged when no off-diagonal entry exceeds `start` times its rotation threshold (a
    // sweep still rotates every pair above the threshold itself), so that sweeps that would only
    // move rounding noise are not started
    if (tid == 0) flags[sweep & 1] = 0;
    jsync(nthr);
    for (int t = tid; t < n * n; t += nthr) {
      const int p = t / n, q = t - (t / n) * n;
      if (p < q) {
        // the rotation test of rot_params at `start` times the thresholds (no rotation
        // parameters)
        const float app = A[p * kLd + p].x, aqq = A[q * kLd + q].x;
        const float2 apq = A[p * kLd + q];
        const float g2 = apq.x * apq.x + apq.y * apq.y;
        const float lim = fmaxf(start * eps * fmaxf(fabsf(app), fabsf(aqq)), start * floor_);
        if (g2 > lim * lim) flags[sweep & 1] = 1;
      }
    }
    jsync(nthr);
    if (!flags[sweep & 1] || sweep >= max_sweeps) break;
    for (int st = 0; st < np - 1; ++st) {
      auto rot_of = [&](int k) -> C4 { return rot_params(A, 2 * k, 2 * k + 1, eps, floor_); };
      if (role == 1) {
        const C b00 = A[p1 * kLd + p2], b01 = A[p1 * kLd + q2];
        const C b10 = A[q1 * kLd + p2], b11 = A[q1 * kLd + q2];
        const C4 ra = rot_of(k1);
        if (k1 == k2) {
          C o00 = b00, o01 = b01, o10 = b10, o11 = b11;
          if (ra.w != R(0)) {
            // a_pp - t|a_pq|, a_qq + t|a_pq|, exact zeros off the diagonal
            o00 = mkc(b00.x - ra.w, R(0));
            o11 = mkc(b11.x + ra.w, R(0));
            o01 = mkc(R(0), R(0));
            o10 = o01;
          }
          An[np1 * kLd + np1] = o00;
          An[np1 * kLd + nq1] = o01;
          An[nq1 * kLd + np1] = o10;
          An[nq1 * kLd + nq1] = o11;
        } else {
          const C4 rb = rot_of(k2);
          const C s1 = mkc(ra.y, ra.z), s2 = mkc(rb.y, rb.z);
          // rows of J1^H B, then (J1^H B) J2; J = [[c, se], [-conj(se), c]]
          const C tp0 = sub_(scl_<C, R>(b00, ra.x), mul_(s1, b10));
          const C tp1 = sub_(scl_<C, R>(b01, ra.x), mul_(s1, b11));
          const C tq0 = add_(mulc_(s1, b00), scl_<C, R>(b10, ra.x));
          const C tq1 = add_(mulc_(s1, b01), scl_<C, R>(b11, ra.x));
          const C o00 = sub_(scl_<C, R>(tp0, rb.x), mul_(tp1, conj_(s2)));
          const C o01 = add_(mul_(tp0, s2), scl_<C, R>(tp1, rb.x));
          const C o10 = sub_(scl_<C, R>(tq0, rb.x), mul_(tq1, conj_(s2)));
          const C o11 = add_(mul_(tq0, s2), scl_<C, R>(tq1, rb.x));
          An[np1 * kLd + np2] = o00;
          An[np1 * kLd + nq2] = o01;
          An[nq1 * kLd + np2] = o10;
          An[nq1 * kLd + nq2] = o11;
          An[np2 * kLd + np1] = conj_(o00);
          An[nq2 * kLd + np1] = conj_(o01);
          An[np2 * kLd + nq1] = conj_(o10);
          An[nq2 * kLd + nq1] = conj_(o11);
        }
      } else if (role == 2) {
        const C vp0 = V[r0 * kLd + p2], vq0 = V[r0 * kLd + q2];
        const C vp1 = V[(r0 + 1) * kLd + p2], vq1 = V[(r0 + 1) * kLd + q2];
        const C4 r = rot_of(k2);
        const C se = mkc(r.y, r.z);
        Vn[r0 * kLd + np2] = sub_(scl_<C, R>(vp0, r.x), mul_(vq0, conj_(se)));
        Vn[r0 * kLd + nq2] = add_(mul_(vp0, se), scl_<C, R>(vq0, r.x));
        Vn[(r0 + 1) * kLd + np2] = sub_(scl_<C, R>(vp1, r.x), mul_(vq1, conj_(se)));
        Vn[(r0 + 1) * kLd + nq2] = add_(mul_(vp1, se), scl_<C, R>(vq1, r.x));
      }
      jsync(nthr);
      C* t = A;
      A = An;
      An = t;
      t = V;
      V = Vn;
      Vn = t;
    }
    ++sweep;
  }
  return sweep;
}

struct alignas(16) EigShared {
  float2 A0[kMaxNc * kLd];   // A0 and A1 are contiguous: the Gram sub-sums use both
  float2 A1[kMaxNc * kLd];
  float2 V[kMaxNc * kLd];
  float2 G[kMaxNc * kLd];
  float2 V1[kMaxNc * kLd];   // second eigenvector buffer of the Jacobi permutation
  float f[kMaxNc];         // sigma''_i / sigma_i
  double lam[kMaxNc];      // eigenvalues
  float sprevf[kMaxNc];    // sigma_prev as float32
  int flags[4];
  int jac_sweeps, jac_odd;   // Jacobi sweeps done; 1 if A and V ended in the second buffers
  float lrs_l1;              // l1 off the prior support of the previous iteration
  unsigned char tri[2][kMaxNc * (kMaxNc + 1) / 2];   // (i, j) of upper-triangle entry e
  double sprev[kMaxNc];    // sigma_prev
  // control scalars read once at entry
  double nuc_prev;
  float sig_prev1;         // nuclear norm of the previous iteration as float (finiteness test)
  float lamL, lamS, haar_max;
  int lambdas_set, rank_prev, sweeps_prev, has_sigma, v_valid;
};


// One chunk sum of a Gram entry over the partials: task = part * nn + e sums partials
// part, part + ksub, part + 2 ksub, ... of entry e, sixteen loads in flight at a time.
// Every partial holds an exactly Hermitian matrix and all entries are summed in the same
// order, so the result is exactly Hermitian too.
__device__ __forceinline__ float2 gram_chunk(const float2* __restrict__ gram_part, int task, int nn, int ksub,
                                             int nparts) {
  const int part = task / nn, e = task - part * nn;
  const float2* src = gram_part + e;
  constexpr int U = 16;
  float sx = 0.f, sy = 0.f;
  for (int p0 = part; p0 < nparts; p0 += ksub * U) {
    float2 v[U];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int pp = p0 + q * ksub;
      v[q] = pp < nparts ? src[(long long)pp * nn] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < U; ++q) {
      sx += v[q].x;
      sy += v[q].y;
    }
  }
  return make_float2(sx, sy);
}

// NCT: the column count fixed at compile time (its loops unroll and their loads pipeline);
// 0 takes it from the geometry at run time.
template <int NCT>
__global__ void __launch_bounds__(kEigThreads, 1) k_eig(const EigArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  EigShared& sh = *reinterpret_cast<EigShared*>(smem_raw);
  DevCtrl* ctrl = a.ctrl;
  const int tid = threadIdx.x;
  const int n = NCT ? NCT : a.g.nc;
  const int np = n + (n & 1);
  // The successor (the data-consistency kernel) is released only after this wait: once it
  // runs, every kernel before this one has completed, so it may read their outputs (X, L and
  // the sparse parts of the previous iteration) before its own wait.
  pdl_wait();   // the Gram partials, statistics and control block come from earlier kernels
  pdl_trigger();
  const int nn = n * n;
  const int nut = n * (n + 1) / 2;
  const bool tol_on = a.tol > 0.0;
  // Every independent global load of the kernel is issued before the first barrier: control
  // scalars, the prior, the previous eigenvectors, the Gram partials and the statistics.
  switch (tid) {
    case 9: sh.flags[2] = ctrl->converged; break;
    case 0: {
      sh.nuc_prev = ctrl->nuclear_cur;
      sh.sig_prev1 = (float)sh.nuc_prev;
    } break;
    case 1: sh.lamL = ctrl->lambda_L; break;
    case 2: sh.lamS = ctrl->lambda_S; break;
    case 3: sh.haar_max = __uint_as_float(ctrl->haar_max_bits); break;
    case 4: sh.lambdas_set = ctrl->lambdas_set; break;
    case 5: sh.rank_prev = ctrl->rank_cur; break;
    case 6: sh.sweeps_prev = ctrl->sweeps_cur; break;
    case 7: sh.has_sigma = a.persist->has_sigma; break;
    case 8: sh.v_valid = a.persist->v_valid; break;
    default: break;
  }
  if (tid >= 32 && tid < 32 + n) {
    const double v = a.sigma_prev[tid - 32];
    sh.sprev[tid - 32] = v;
    sh.sprevf[tid - 32] = (float)v;
  }
  if (!a.finalize) {
    const float2* vsrc = a.Vin ? a.Vin : a.V;
    for (int e = tid; e < nn; e += kEigThreads) sh.V[(e / n) * kLd + e % n] = vsrc[e];
  }
  // statistics of iteration iter-1: the last warp sums the data-consistency partials (x:
  // ||E Z - d||^2, z: ||Z_k - Z_{k-1}||^2, w: ||Z_{k-1}||^2), the warp before it the sparse
  // step's l1 off the prior support; eight loads per lane are in flight at a time
  const bool stats_on = a.iter > 1 && a.part != 2;
  const int sw = (kEigThreads >> 5) - 1;
  float4 st4 = make_float4(0.f, 0.f, 0.f, 0.f);
  if (stats_on && (tid >> 5) == sw) {
    const int lane = tid & 31;
    const float4* dc4 = reinterpret_cast<const float4*>(a.dc_part);
    for (int i0 = 0; i0 < a.ndc; i0 += 256) {
      float4 q[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int i = i0 + lane + 32 * u;
        q[u] = i < a.ndc ? dc4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        st4.x += q[u].x;
        st4.z += q[u].y;
        st4.w += q[u].z;
      }
    }
  } else if (stats_on && (tid >> 5) == sw - 1) {
    const int lane = tid & 31;
    float l1 = 0.f;
    for (int i0 = 0; i0 < a.lrs_parts; i0 += 256) {
      float q[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int i = i0 + lane + 32 * u;
        q[u] = i < a.lrs_parts ? a.lrs_part[2 * i] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) l1 += q[u];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l1 += __shfl_xor_sync(0xffffffffu, l1, o);
    if (lane == 0) sh.lrs_l1 = l1;
  }
  // Gram partials: all n x n entries, ksub interleaved chunks per entry
  const int ksub = nn <= kEigThreads / 2 ? 2 : 1;
  float2* sub = sh.A0;   // scratch [ksub][nn], spans A0 and A1 (free until the Jacobi)
  // at most two tasks per thread: ksub * nn <= 2 * kEigThreads (n <= 32)
  float2 gacc0 = make_float2(0.f, 0.f), gacc1 = make_float2(0.f, 0.f);
  if (!a.finalize && a.part != 2) {
    gacc0 = gram_chunk(a.gram_part, tid, nn, ksub, a.nparts);
    if (tid + kEigThreads < ksub * nn) gacc1 = gram_chunk(a.gram_part, tid + kEigThreads, nn, ksub, a.nparts);
  }
  if (tid < n) {
    int e = tid * n - tid * (tid - 1) / 2;
    for (int j = tid; j < n; ++j, ++e) {
      sh.tri[0][e] = (unsigned char)tid;
      sh.tri[1][e] = (unsigned char)j;
    }
  }
  __syncthreads();
  if (sh.flags[2]) return;

  // 1. statistics record and the stopping rule (the second part of the float64 mode has done it)
  if (stats_on && (tid >> 5) == sw) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      st4.x += __shfl_xor_sync(0xffffffffu, st4.x, o);
      st4.y += __shfl_xor_sync(0xffffffffu, st4.y, o);
      st4.z += __shfl_xor_sync(0xffffffffu, st4.z, o);
      st4.w += __shfl_xor_sync(0xffffffffu, st4.w, o);
    }
    if ((tid & 31) == 0) {
      const float r2 = st4.x, l1 = sh.lrs_l1;
      const float rel = sqrtf(st4.z / fmaxf(st4.w, 1e-30f));
      const bool nonfinite = !isfinite(r2) || !isfinite(l1) || !isfinite(sh.sig_prev1);
      const bool stop = nonfinite || (tol_on && rel < a.tol_f);
      const double nuc = sh.nuc_prev;
      IterRec& rec = a.hist[a.iter - 2];
      rec.resid2 = r2;
      rec.nuclear = nuc;
      rec.l1 = l1;
      rec.rel_change = rel;
      rec.rank = sh.rank_prev;
      rec.sweeps = sh.sweeps_prev;
      ctrl->iters_done = a.iter - 1;
      if (nonfinite) ctrl->err |= kErrNonfinite;
      if (stop) ctrl->converged = 1;
      sh.flags[3] = stop;
    }
  }
  if (a.finalize) return;
  if (tol_on && stats_on) {
    __syncthreads();
    if (sh.flags[3]) return;
  }

  int sweeps = 0;
  float2* Af = sh.A0;    // eigenvalues on the diagonal after the Jacobi
  float2* Vres = sh.V;   // eigenvectors (columns)
  if (a.part != 2) {
    // 2. Gram matrix: combine the chunk sums in a fixed order; exact Hermitian symmetry
    if (tid < ksub * nn) sub[tid] = gacc0;
    if (tid + kEigThreads < ksub * nn) sub[tid + kEigThreads] = gacc1;
    const bool warm = sh.v_valid != 0;
    if (!warm)
      for (int e = tid; e < nn; e += kEigThreads) {
        const int i = e / n, j = e - i * n;
        sh.V[i * kLd + j] = (i == j) ? make_float2(1.f, 0.f) : make_float2(0.f, 0.f);
      }
    for (int e = tid; e < np * np; e += kEigThreads) {
      const int i = e / np, j = e - (e / np) * np;
      if (i >= n || j >= n) sh.V[i * kLd + j] = (i == j) ? make_float2(1.f, 0.f) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int e = tid; e < nn; e += kEigThreads) {
      const int i = e / n, j = e - i * n;
      float2 s = sub[e];
      for (int q = 1; q < ksub; ++q) s = cadd(s, sub[q * nn + e]);
      if (i == j) s.y = 0.f;
      sh.G[i * kLd + j] = s;
    }
    __syncthreads();

    // 3. Jacobi, warm-started from the previous eigenvectors
    if (warm) {
      // A1 = G V, then A0 = V^H A1 (upper triangle, mirrored: exactly Hermitian)
      for (int e = tid; e < nn; e += kEigThreads) {
        const int i = e / n, j = e - (e / n) * n;
        float2 s = make_float2(0.f, 0.f);
#pragma unroll 8
        for (int k = 0; k < n; ++k) s = cadd(s, cmul(sh.G[i * kLd + k], sh.V[k * kLd + j]));
        sh.A1[i * kLd + j] = s;
      }
      __syncthreads();
      for (int e = tid; e < nut; e += kEigThreads) {
        const int i = sh.tri[0][e], j = sh.tri[1][e];
        float2 s = make_float2(0.f, 0.f);
#pragma unroll 8
        for (int k = 0; k < n; ++k) s = cadd(s, cmulc(sh.V[k * kLd + i], sh.A1[k * kLd + j]));
        if (i == j) s.y = 0.f;
        sh.A0[i * kLd + j] = s;
        sh.A0[j * kLd + i] = cconj(s);
      }
    } else {
      for (int e = tid; e < nut; e += kEigThreads) {
        const int i = sh.tri[0][e], j = sh.tri[1][e];
        const float2 g = sh.G[i * kLd + j];
        sh.A0[i * kLd + j] = g;
        sh.A0[j * kLd + i] = cconj(g);
      }
    }
    for (int e = tid; e < np * np; e += kEigThreads) {
      const int i = e / np, j = e - (e / np) * np;
      if (i >= n || j >= n) sh.A0[i * kLd + j] = make_float2(0.f, 0.f);
    }
    __syncthreads();
    float trace = 0.f;
#pragma unroll 8
    for (int i = 0; i < n; ++i) trace += fabsf(sh.A0[i * kLd + i].x);
    float2* Afn = sh.A1;
    float2* Vf = sh.V;
    float2* Vfn = sh.V1;
    if (tid < jacobi_threads(n)) {
      // a new sweep starts above 8x the rotation threshold (64u of the larger diagonal entry or
      // 8u of the trace), still below the float32 Gram's own accumulation error (about
      // u sqrt(rows) of the trace); before the float64 refinement (part 1) at 2x, which leaves
      // the refinement pairs coupled well below its 1e-3 gap limit
      sweeps = jacobi<NCT>(Af, Afn, Vf, Vfn, n, 4.8e-7f, 6.0e-8f * trace + 1e-30f, 12, a.part == 1 ? 2.f : 8.f,
                           sh.flags);
      if (tid == 0) {
        // own fields: other Jacobi threads may still read flags[] in their last convergence test
        sh.jac_sweeps = sweeps;
        sh.jac_odd = Af != sh.A0;   // the results sit in the second buffers (odd step count)
      }
    }
    __syncthreads();
    sweeps = sh.jac_sweeps;
    if (sh.jac_odd) {
      Af = sh.A1;
      Vres = sh.V1;
    }

    if (a.part == 1) {
      // float64 mode, first part: hand the Gram, the float32 eigenvectors and eigenvalues to the
      // float64 Rayleigh-Ritz kernels (k_ritz64_a, k_ritz64_b)
      for (int e = tid; e < nn; e += kEigThreads) {
        const int i = e / n, j = e - (e / n) * n;
        a.Gout[e] = sh.G[i * kLd + j];
        a.V[e] = Vres[i * kLd + j];
      }
      for (int i = tid; i < n; i += kEigThreads) a.lam64[i] = (double)Af[i * kLd + i].x;
      if (tid == 32) ctrl->sweeps_cur = sweeps;
      return;
    }
    // float32 path: warp 0 reads the eigenvalues from the diagonal of Af below
  } else {
    // float64 mode, second part: the Rayleigh-Ritz eigenvalues and refined eigenvectors
    // (V was loaded with the warm start above)
    for (int i = tid; i < n; i += kEigThreads) sh.lam[i] = a.lam64[i];
    __syncthreads();
  }

  // 4. singular values, thresholds, prior pull, rank guard: warp 0, lane i = eigenvalue i
  //    (n <= 32), ranks and sums by shuffles; in float64 after the float64 refinement, in
  //    float32 otherwise (float64 issues at a small fraction of the float32 rate here).
  if (tid < 32) {
    const int i = tid;
    const bool act = i < n;
    const unsigned full = 0xffffffffu;
    double s2d = 0.0;
    int r = 0;
    if (a.eig_fp64) {
      const double li = act ? sh.lam[i] : -1.0e300;
      for (int j = 0; j < n; ++j) {
        const double lj = __shfl_sync(full, li, j);
        r += (lj > li) || (lj == li && j < i);
      }
      const double s = act ? sqrt(fmax(li, 0.0)) : 0.0;
      double sig1 = s;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sig1 = fmax(sig1, __shfl_xor_sync(full, sig1, o));
      if (a.iter == 1 && !sh.lambdas_set) {
        sh.lamL = (float)(a.lambda_L_rel * sig1);
        sh.lamS = (float)(a.lambda_S_rel * (double)sh.haar_max);
        if (i == 0) {
          ctrl->lambda_L = sh.lamL;
          ctrl->lambda_S = sh.lamS;
          ctrl->sigma_max = sig1;
          ctrl->lambdas_set = 1;
        }
      }
      __syncwarp();
      if (act) {
        const double s1 = fmax(s - (double)sh.lamL, 0.0);
        s2d = sh.has_sigma ? s1 - a.lambda_p * (s1 - sh.sprev[r]) : s1;
        if (s <= a.rank_tau * sig1) s2d = 0.0;
        sh.f[i] = s > 0.0 ? (float)(s2d / s) : 0.f;
      }
    } else {
      // float32: every lane reads all eigenvalues from shared memory (broadcast loads in
      // flight together) for its rank and the largest eigenvalue; selects instead of
      // branches; float32 copies of sigma_prev, lambda_p and tau
      const float li = act ? Af[i * kLd + i].x : -3.0e38f;
      float lmax = -3.0e38f;
#pragma unroll 8
      for (int j = 0; j < n; ++j) {
        const float lj = Af[j * kLd + j].x;
        r += (int)(lj > li) | ((int)(lj == li) & (int)(j < i));
        lmax = fmaxf(lmax, lj);
      }
      // sqrt is monotone and correctly rounded: max_i sqrt(l_i) = sqrt(max_i l_i)
      const float s = act ? sqrtf(fmaxf(li, 0.f)) : 0.f;
      const float sig1 = sqrtf(fmaxf(lmax, 0.f));
      if (a.iter == 1 && !sh.lambdas_set) {
        sh.lamL = (float)(a.lambda_L_rel * (double)sig1);
        sh.lamS = (float)(a.lambda_S_rel * (double)sh.haar_max);
        if (i == 0) {
          ctrl->lambda_L = sh.lamL;
          ctrl->lambda_S = sh.lamS;
          ctrl->sigma_max = (double)sig1;
          ctrl->lambdas_set = 1;
        }
      }
      __syncwarp();
      const float s1 = fmaxf(s - sh.lamL, 0.f);
      const float sp = sh.sprevf[act ? r : 0];
      float s2 = sh.has_sigma ? s1 - a.lambda_p_f * (s1 - sp) : s1;
      s2 = (s <= a.rank_tau_f * sig1 || !act) ? 0.f : s2;
      const float fi = s > 0.f ? s2 / s : 0.f;
      if (act) sh.f[i] = fi;
      s2d = (double)s2;
    }
    if (act) a.sigma_out[r] = s2d;   // sigma'' in rank order
    const int rk = __popc(__ballot_sync(full, s2d > 0.0));
    double nuc;
    if (a.eig_fp64) {
      nuc = s2d;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) nuc += __shfl_xor_sync(full, nuc, o);
    } else {
      float nf = (float)s2d;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) nf += __shfl_xor_sync(full, nf, o);
      nuc = (double)nf;
    }
    if (i == 0) {
      ctrl->nuclear_cur = nuc;
      ctrl->rank_cur = rk;
      if (a.part != 2) ctrl->sweeps_cur = sweeps;
    }
  }
  __syncthreads();
  // 5. W = V diag(f) V^H and the eigenvectors for the next warm start
  for (int e = tid; e < nn; e += kEigThreads) {
    const int i = e / n, j = e - (e / n) * n;
    float2 s = make_float2(0.f, 0.f);
#pragma unroll 8
    for (int k = 0; k < n; ++k) {
      // f_k = 0 contributes exactly nothing (terms are not formed for it)
      const float fk = sh.f[k];
      const float2 t = cscale(cmul(Vres[i * kLd + k], cconj(Vres[j * kLd + k])), fk);
      s = fk != 0.f ? cadd(s, t) : s;
    }
    a.W[i * n + j] = s;
    a.V[i * n + j] = Vres[i * kLd + j];
  }
  if (tid == 0) a.persist->v_valid = 1;
}



template <int NCT>
static cudaError_t launch_eig_n(const EigArgs& a, cudaStream_t st) {
  const size_t smem = sizeof(EigShared);
  static bool attr_set = false;
  if (smem > 48 * 1024 && !attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_eig<NCT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  cudaError_t e = launch_pdl(k_eig<NCT>, dim3(1), dim3(kEigThreads), smem, st, a);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_eig(const EigArgs& a, cudaStream_t st) {
  switch (a.g.nc) {
    case 8: return launch_eig_n<8>(a, st);
    case 16: return launch_eig_n<16>(a, st);
    case 32: return launch_eig_n<32>(a, st);
    default: return launch_eig_n<0>(a, st);
  }
}

// float64 Rayleigh-Ritz refinement of the float32 eigendecomposition (LPS_EIG_FP64), one CTA of
// four warps per eigenvector j, in two kernels (the second needs the diagonal of A):
//   k_ritz64_a: A[:, j] = V^H (G v_j)
//   k_ritz64_b: lambda_j = A_jj + sum_i |A_ij|^2 / (A_jj - A_ii) and
//               v'_j = v_j + sum_i v_i A_ij / (A_jj - A_ii), normalised,
// the first- and second-order corrections of the eigenpairs of A = D + F (F the off-diagonal
// part left by the float32 Jacobi, ~1e-7 |A|), taken only for pairs whose coupling is below
// 1e-3 of their gap, where the corrected vectors stay orthonormal to ~1e-6; inside a cluster of
// close eigenvalues (the noise floor) any rotation of the vectors is an eigenbasis to the
// cluster's width, so the float32 vectors, orthonormal to float32 rounding, are kept there.
// Sums over k are split over the four warps (a quarter of k each) and added in a fixed order.
constexpr int kRitzThreads = 128;

// s_w[i] = sum over k in quarter w of f(i, k), then out[i] = s_0 + s_1 + s_2 + s_3 (warp 0).
template <typename F>
__device__ __forceinline__ double2 ritz_sum(int n, F f, double2 (&part)[4][kMaxNc]) {
  const int i = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int kc = (n + 3) / 4, k0 = w * kc, k1 = min(n, k0 + kc);
  double2 s = make_double2(0.0, 0.0);
  if (i < n)
    for (int k = k0; k < k1; ++k) s = add_(s, f(i, k));
  part[w][i] = s;
  __syncthreads();
  return add_(add_(part[0][i], part[1][i]), add_(part[2][i], part[3][i]));
}

__global__ void __launch_bounds__(kRitzThreads) k_ritz64_a(const RitzArgs a) {
  pdl_trigger();
  pdl_wait();
  if (a.ctrl->converged) return;
  __shared__ float2 Vs[kMaxNc * kMaxNc];
  __shared__ float2 Gs[kMaxNc * kMaxNc];
  __shared__ double2 part[4][kMaxNc];
  __shared__ double2 t[kMaxNc];
  const int n = a.n, j = blockIdx.x, tid = threadIdx.x;
  for (int q = tid; q < n * n; q += kRitzThreads) {
    Vs[q] = a.V[q];
    Gs[q] = a.G[q];
  }
  __syncthreads();
  // t = G v_j
  const double2 gv = ritz_sum(n, [&](int i, int k) {
    const float2 g = Gs[i * n + k], v = Vs[k * n + j];
    return mul_(make_double2(g.x, g.y), make_double2(v.x, v.y));
  }, part);
  if (tid < n) t[tid] = gv;
  __syncthreads();
  // A_ij = sum_k conj(V_ki) t_k
  const double2 aij = ritz_sum(n, [&](int i, int k) {
    const float2 v = Vs[k * n + i];
    return mulc_(make_double2(v.x, v.y), t[k]);
  }, part);
  if (tid < n) a.A[tid * n + j] = aij;
}

__global__ void __launch_bounds__(kRitzThreads) k_ritz64_b(const RitzArgs a) {
  pdl_trigger();
  pdl_wait();
  if (a.ctrl->converged) return;
  __shared__ float2 Vs[kMaxNc * kMaxNc];
  __shared__ double2 part[4][kMaxNc];
  __shared__ double2 e[kMaxNc];
  __shared__ double dls[kMaxNc];
  const int n = a.n, j = blockIdx.x, tid = threadIdx.x;
  for (int q = tid; q < n * n; q += kRitzThreads) Vs[q] = a.V[q];
  const double ajj = a.A[j * n + j].x;
  if (tid < kMaxNc) {
    const int i = tid;
    double2 c = make_double2(0.0, 0.0);
    double dl = 0.0;
    if (i < n && i != j) {
      const double2 aij = a.A[i * n + j];
      const double gap = ajj - a.A[i * n + i].x;
      const double m2 = aij.x * aij.x + aij.y * aij.y;
      if (m2 < 1e-6 * gap * gap) {   // |E_ij| < 1e-3: the dropped second-order terms stay below 1e-6
        c = make_double2(aij.x / gap, aij.y / gap);
        dl = m2 / gap;
      }
    }
    e[i] = c;
    dls[i] = dl;
  }
  __syncthreads();
  // v'_j row i: v_ij + sum_k v_ik e_k
  double2 v = ritz_sum(n, [&](int i, int k) {
    const float2 vik = Vs[i * n + k];
    return mul_(make_double2(vik.x, vik.y), e[k]);
  }, part);
  if (tid >= 32) return;
  const int i = tid;
  double dl = dls[i];
  if (i < n) {
    const float2 vij = Vs[i * n + j];
    v = add_(make_double2(vij.x, vij.y), v);
  } else {
    v = make_double2(0.0, 0.0);
  }
  double nrm = v.x * v.x + v.y * v.y;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    dl += __shfl_xor_sync(0xffffffffu, dl, o);
  }
  const double inv = nrm > 0.0 ? 1.0 / sqrt(nrm) : 1.0;
  if (i < n) a.Vout[i * n + j] = make_float2((float)(v.x * inv), (float)(v.y * inv));
  if (i == 0) a.lam64[j] = ajj + dl;
}

cudaError_t launch_ritz64(const RitzArgs& a, cudaStream_t st) {
  if (a.n > kMaxNc) return cudaErrorInvalidValue;
  cudaError_t e = launch_pdl(k_ritz64_a, dim3(a.n), dim3(kRitzThreads), 0, st, a);
  if (e != cudaSuccess) return e;
  e = launch_pdl(k_ritz64_b, dim3(a.n), dim3(kRitzThreads), 0, st, a);
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace lps
