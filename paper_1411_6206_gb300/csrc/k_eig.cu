// Steps (1) and (2) of Algorithm 1 (Sec. 3) on the small side of the Casorati matrix.
//
// The singular values and right singular vectors of M = X - S (N_r x nc, N_r >> nc) are
// those of its Gram matrix G = M^H M = V diag(sigma^2) V^H. One CTA:
//   1. records the statistics of the previous iteration (residual, nuclear norm, l1 off the
//      prior support, objective, relative change) and applies the stopping rule (Sec. 3:
//      stop when the relative change of the solution falls below the tolerance);
//   2. sums the per-plane Gram partials in a fixed order (compensated float32);
//   3. diagonalises G by cyclic two-sided Jacobi rotations in round-robin order (nc/2
//      disjoint rotations per step, one barrier per step), warm-started from the previous
//      iteration's eigenvectors; optionally polished by float64 Jacobi sweeps;
//   4. sigma = sqrt(lambda), step (1) sigma' = max(sigma - lambda_L, 0), step (2)
//      sigma'' = sigma' - lambda_p (sigma' - sigma_prev) (matched by rank), rank guard
//      sigma''_i = 0 where sigma_i <= tau sigma_1, in float64;
//   5. writes W = V diag(sigma''/sigma) V^H so that L = M W = U diag(sigma'') V^H.
// At the first iteration it also fixes lambda_L = rel_L sigma_1(X_0) and
// lambda_S = rel_S max|T(X_0)|.
#include "lps_internal.cuh"

namespace lps {

constexpr int kEigThreads = 256;
constexpr int kLd = kMaxNc + 1;   // leading dimension of the shared matrices

template <typename R>
struct Cx;
template <>
struct Cx<float> {
  using T = float2;
};
template <>
struct Cx<double> {
  using T = double2;
};

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

// Round-robin pairing: at step s of a sweep over np (even) indices, pair k is (p, q).
__device__ __forceinline__ void rr_pair(int np, int s, int k, int& p, int& q) {
  const int m = np - 1;
  if (k == 0) {
    p = m;
    q = s;
  } else {
    p = (s + k) % m;
    q = (s - k + m) % m;
  }
}

template <typename R>
struct Rot {
  R c, s;
  typename Cx<R>::T e;   // unit phase of a_pq
  R t, gabs;
  bool on;
};

template <typename R>
__device__ __forceinline__ Rot<R> rot_params(const typename Cx<R>::T* A, int p, int q, R eps_rel, R abs_floor) {
  using C = typename Cx<R>::T;
  Rot<R> r;
  const R app = A[p * kLd + p].x, aqq = A[q * kLd + q].x;
  const C apq = A[p * kLd + q];
  const R g = sqrt(apq.x * apq.x + apq.y * apq.y);
  const R lim = fmax(eps_rel * sqrt(fabs(app * aqq)), abs_floor);
  r.on = g > lim;
  if (r.on) {
    const R tau = (aqq - app) / (R(2) * g);
    const R t = (tau >= R(0) ? R(1) : R(-1)) / (fabs(tau) + sqrt(R(1) + tau * tau));
    r.c = R(1) / sqrt(R(1) + t * t);
    r.s = t * r.c;
    r.e = mkc(apq.x / g, apq.y / g);
    r.t = t;
    r.gabs = g;
  } else {
    r.c = R(1);
    r.s = R(0);
    r.e = mkc(R(1), R(0));
    r.t = R(0);
    r.gabs = g;
  }
  return r;
}

// Cyclic Jacobi on the Hermitian n x n matrix in A[0] (padded to even np with a zero
// row/column); eigenvectors accumulated into V. Returns the sweeps done.
template <typename R>
__device__ int jacobi(typename Cx<R>::T* A0, typename Cx<R>::T* A1, typename Cx<R>::T* V, int n, R eps_rel,
                      R abs_floor, int max_sweeps, int* flags, typename Cx<R>::T** result) {
  using C = typename Cx<R>::T;
  const int np = n + (n & 1);
  const int nh = np >> 1;
  const int nblk = nh * (nh + 1) / 2;
  const int ntask = nblk + np * nh;
  C* Ac = A0;
  C* An = A1;
  if (threadIdx.x == 0) flags[0] = flags[1] = flags[2] = 0;
  __syncthreads();
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) flags[(sweep + 1) % 3] = 0;
    for (int st = 0; st < np - 1; ++st) {
      for (int t = threadIdx.x; t < ntask; t += blockDim.x) {
        if (t < nblk) {
          // upper-triangular pair block (k1 <= k2)
          int k1 = 0, rem = t;
          while (rem >= nh - k1) {
            rem -= nh - k1;
            ++k1;
          }
          const int k2 = k1 + rem;
          int p1, q1, p2, q2;
          rr_pair(np, st, k1, p1, q1);
          rr_pair(np, st, k2, p2, q2);
          const Rot<R> r1 = rot_params<R>(Ac, p1, q1, eps_rel, abs_floor);
          if (r1.on) flags[sweep % 3] = 1;
          if (k1 == k2) {
            if (r1.on) {
              An[p1 * kLd + p1] = mkc(Ac[p1 * kLd + p1].x - r1.t * r1.gabs, R(0));
              An[q1 * kLd + q1] = mkc(Ac[q1 * kLd + q1].x + r1.t * r1.gabs, R(0));
              An[p1 * kLd + q1] = mkc(R(0), R(0));
              An[q1 * kLd + p1] = mkc(R(0), R(0));
            } else {
              An[p1 * kLd + p1] = Ac[p1 * kLd + p1];
              An[q1 * kLd + q1] = Ac[q1 * kLd + q1];
              An[p1 * kLd + q1] = Ac[p1 * kLd + q1];
              An[q1 * kLd + p1] = Ac[q1 * kLd + p1];
            }
            continue;
          }
          const Rot<R> r2 = rot_params<R>(Ac, p2, q2, eps_rel, abs_floor);
          const C bpp = Ac[p1 * kLd + p2], bpq = Ac[p1 * kLd + q2];
          const C bqp = Ac[q1 * kLd + p2], bqq = Ac[q1 * kLd + q2];
          // rows: J1^H B
          const C se1 = scl_<C, R>(r1.e, r1.s);           // s1 e1
          const C se1c = conj_(se1);                      // s1 conj(e1)
          const C rpp = sub_(scl_<C, R>(bpp, r1.c), mul_(se1, bqp));
          const C rpq = sub_(scl_<C, R>(bpq, r1.c), mul_(se1, bqq));
          const C rqp = add_(mul_(se1c, bpp), scl_<C, R>(bqp, r1.c));
          const C rqq = add_(mul_(se1c, bpq), scl_<C, R>(bqq, r1.c));
          // columns: (J1^H B) J2
          const C se2 = scl_<C, R>(r2.e, r2.s);
          const C se2c = conj_(se2);
          const C opp = sub_(scl_<C, R>(rpp, r2.c), mul_(rpq, se2c));
          const C opq = add_(mul_(rpp, se2), scl_<C, R>(rpq, r2.c));
          const C oqp = sub_(scl_<C, R>(rqp, r2.c), mul_(rqq, se2c));
          const C oqq = add_(mul_(rqp, se2), scl_<C, R>(rqq, r2.c));
          An[p1 * kLd + p2] = opp;
          An[p1 * kLd + q2] = opq;
          An[q1 * kLd + p2] = oqp;
          An[q1 * kLd + q2] = oqq;
          An[p2 * kLd + p1] = conj_(opp);
          An[q2 * kLd + p1] = conj_(opq);
          An[p2 * kLd + q1] = conj_(oqp);
          An[q2 * kLd + q1] = conj_(oqq);
        } else {
          const int vt = t - nblk;
          const int i = vt / nh, k = vt - (vt / nh) * nh;
          int p, q;
          rr_pair(np, st, k, p, q);
          const Rot<R> r = rot_params<R>(Ac, p, q, eps_rel, abs_floor);
          if (r.on) {
            const C vp = V[i * kLd + p], vq = V[i * kLd + q];
            const C se = scl_<C, R>(r.e, r.s);
            V[i * kLd + p] = sub_(scl_<C, R>(vp, r.c), mul_(vq, conj_(se)));
            V[i * kLd + q] = add_(mul_(vp, se), scl_<C, R>(vq, r.c));
          }
        }
      }
      __syncthreads();
      C* tmp = Ac;
      Ac = An;
      An = tmp;
    }
    const int any = flags[sweep % 3];
    if (!any) {
      ++sweep;
      break;
    }
  }
  *result = Ac;
  return sweep;
}

__device__ __forceinline__ double block_sum_d(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += red[i];
  __syncthreads();
  if (threadIdx.x == 0) red[0] = r;
  __syncthreads();
  r = red[0];
  __syncthreads();
  return r;
}

struct alignas(16) EigShared {
  float2 A0[kMaxNc * kLd];
  float2 A1[kMaxNc * kLd];
  float2 V[kMaxNc * kLd];
  float2 G[kMaxNc * kLd];
  double lam[kMaxNc];
  double f[kMaxNc];
  int rank[kMaxNc];
  int flags[4];
  double red[32];
  float2* Aout;
};

struct alignas(16) EigShared64 {
  double2 A0[kMaxNc * kLd];
  double2 A1[kMaxNc * kLd];
  double2 V[kMaxNc * kLd];
  double2 T[kMaxNc * kLd];
  double2* Aout;
};

__global__ void __launch_bounds__(kEigThreads, 1) k_eig(const EigArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  EigShared& sh = *reinterpret_cast<EigShared*>(smem_raw);
  DevCtrl* ctrl = a.ctrl;
  if (ctrl->converged) return;
  const int tid = threadIdx.x;
  const int n = a.g.nc;

  // 1. statistics of iteration iter-1 and the stopping rule
  if (a.iter > 1) {
    double r2 = 0.0;
    for (int i = tid; i < a.g.nx; i += kEigThreads) r2 += (double)a.dc_part[i];
    double l1 = 0.0, dz2 = 0.0, z2 = 0.0;
    for (int i = tid; i < a.g.ntiles; i += kEigThreads) {
      l1 += (double)a.lrs_part[i * 4 + 0];
      dz2 += (double)a.lrs_part[i * 4 + 1];
      z2 += (double)a.lrs_part[i * 4 + 2];
    }
    r2 = block_sum_d(r2, sh.red);
    l1 = block_sum_d(l1, sh.red);
    dz2 = block_sum_d(dz2, sh.red);
    z2 = block_sum_d(z2, sh.red);
    const double rel = sqrt(dz2 / fmax(z2, 1e-300));
    const double nuc = ctrl->nuclear_cur;
    const bool nonfinite = !isfinite(r2) || !isfinite(nuc) || !isfinite(l1);
    if (tid == 0) {
      IterRec& rec = a.hist[a.iter - 2];
      rec.resid2 = r2;
      rec.nuclear = nuc;
      rec.l1 = l1;
      rec.objective = 0.5 * r2 + (double)ctrl->lambda_L * nuc + (double)ctrl->lambda_S * l1;
      rec.rel_change = rel;
      rec.rank = ctrl->rank_cur;
      ctrl->iters_done = a.iter - 1;
      if (nonfinite) {
        ctrl->err |= kErrNonfinite;
        ctrl->converged = 1;
      } else if (a.tol > 0.0 && rel < a.tol) {
        ctrl->converged = 1;
      }
    }
    if (a.finalize || nonfinite || (a.tol > 0.0 && rel < a.tol)) return;
  }
  if (a.finalize) return;

  // 2. Gram matrix from the per-plane partials (compensated sums, fixed order)
  const int nn = n * n;
  for (int e = tid; e < nn; e += kEigThreads) {
    float sx = 0.f, sy = 0.f, cx = 0.f, cy = 0.f;
    for (int p = 0; p < a.nparts; ++p) {
      const float2 v = a.gram_part[(long long)p * nn + e];
      const float yx = v.x - cx, yy = v.y - cy;
      const float tx = sx + yx, ty = sy + yy;
      cx = (tx - sx) - yx;
      cy = (ty - sy) - yy;
      sx = tx;
      sy = ty;
    }
    const int i = e / n, j = e - (e / n) * n;
    if (i == j) sy = 0.f;
    sh.G[i * kLd + j] = make_float2(sx, sy);
  }
  __syncthreads();

  // 3. Jacobi, warm-started from the previous eigenvectors
  const int np = n + (n & 1);
  const bool warm = ctrl->v_valid != 0;
  for (int e = tid; e < np * np; e += kEigThreads) {
    const int i = e / np, j = e - (e / np) * np;
    float2 vv = (i == j) ? make_float2(1.f, 0.f) : make_float2(0.f, 0.f);
    if (warm && i < n && j < n) vv = a.V[i * n + j];
    sh.V[i * kLd + j] = vv;
  }
  __syncthreads();
  if (warm) {
    // A1 = G V, then A0 = V^H A1
    for (int e = tid; e < n * n; e += kEigThreads) {
      const int i = e / n, j = e - (e / n) * n;
      float2 s = make_float2(0.f, 0.f);
      for (int k = 0; k < n; ++k) s = cadd(s, cmul(sh.G[i * kLd + k], sh.V[k * kLd + j]));
      sh.A1[i * kLd + j] = s;
    }
    __syncthreads();
    for (int e = tid; e < n * n; e += kEigThreads) {
      const int i = e / n, j = e - (e / n) * n;
      float2 s = make_float2(0.f, 0.f);
      for (int k = 0; k < n; ++k) s = cadd(s, cmulc(sh.V[k * kLd + i], sh.A1[k * kLd + j]));
      sh.A0[i * kLd + j] = s;
    }
    __syncthreads();
    // exact Hermitian symmetry: keep the upper triangle, real diagonal
    for (int e = tid; e < n * n; e += kEigThreads) {
      const int i = e / n, j = e - (e / n) * n;
      if (i < j) sh.A0[j * kLd + i] = cconj(sh.A0[i * kLd + j]);
      if (i == j) sh.A0[i * kLd + i].y = 0.f;
    }
  } else {
    for (int e = tid; e < n * n; e += kEigThreads) {
      const int i = e / n, j = e - (e / n) * n;
      sh.A0[i * kLd + j] = sh.G[i * kLd + j];
    }
  }
  for (int e = tid; e < np * np; e += kEigThreads) {
    const int i = e / np, j = e - (e / np) * np;
    if (i >= n || j >= n) sh.A0[i * kLd + j] = make_float2(0.f, 0.f);
  }
  __syncthreads();
  float trace = 0.f;
  for (int i = 0; i < n; ++i) trace += fabsf(sh.A0[i * kLd + i].x);
  float2* Af = nullptr;
  jacobi<float>(sh.A0, sh.A1, sh.V, n, 2.0e-7f, 1.0e-9f * trace, 16, sh.flags, &Af);
  __syncthreads();

  if (a.eig_fp64) {
    // Float64 polish: A = V^H G V in double, then double Jacobi sweeps; V <- V Q.
    EigShared64& d = *reinterpret_cast<EigShared64*>(smem_raw + sizeof(EigShared));
    for (int e = tid; e < np * np; e += kEigThreads) {
      const int i = e / np, j = e - (e / np) * np;
      const float2 v = sh.V[i * kLd + j];
      d.V[i * kLd + j] = make_double2(v.x, v.y);
    }
    __syncthreads();
    for (int e = tid; e < n * n; e += kEigThreads) {
      const int i = e / n, j = e - (e / n) * n;
      double2 s = make_double2(0.0, 0.0);
      for (int k = 0; k < n; ++k) {
        const float2 gk = sh.G[i * kLd + k];
        s = add_(s, mul_(make_double2(gk.x, gk.y), d.V[k * kLd + j]));
      }
      d.T[i * kLd + j] = s;
    }
    __syncthreads();
    for (int e = tid; e < np * np; e += kEigThreads) {
      const int i = e / np, j = e - (e / np) * np;
      double2 s = make_double2(0.0, 0.0);
      if (i < n && j < n)
        for (int k = 0; k < n; ++k) s = add_(s, mulc_(d.V[k * kLd + i], d.T[k * kLd + j]));
      d.A0[i * kLd + j] = s;
    }
    __syncthreads();
    for (int e = tid; e < n * n; e += kEigThreads) {
      const int i = e / n, j = e - (e / n) * n;
      if (i < j) d.A0[j * kLd + i] = conj_(d.A0[i * kLd + j]);
      if (i == j) d.A0[i * kLd + i].y = 0.0;
    }
    __syncthreads();
    double tr = 0.0;
    for (int i = 0; i < n; ++i) tr += fabs(d.A0[i * kLd + i].x);
    double2* Ad = nullptr;
    jacobi<double>(d.A0, d.A1, d.V, n, 1.0e-15, 1.0e-17 * tr, 8, sh.flags, &Ad);
    __syncthreads();
    for (int i = tid; i < n; i += kEigThreads) sh.lam[i] = Ad[i * kLd + i].x;
    for (int e = tid; e < np * np; e += kEigThreads) {
      const int i = e / np, j = e - (e / np) * np;
      const double2 v = d.V[i * kLd + j];
      sh.V[i * kLd + j] = make_float2((float)v.x, (float)v.y);
    }
  } else {
    for (int i = tid; i < n; i += kEigThreads) sh.lam[i] = (double)Af[i * kLd + i].x;
  }
  __syncthreads();

  // 4. singular values, thresholds, prior pull, rank guard (float64 scalars)
  double sig1 = 0.0;
  for (int i = 0; i < n; ++i) sig1 = fmax(sig1, sqrt(fmax(sh.lam[i], 0.0)));
  if (tid == 0 && a.iter == 1 && !ctrl->lambdas_set) {
    ctrl->lambda_L = (float)(a.lambda_L_rel * sig1);
    ctrl->lambda_S = (float)(a.lambda_S_rel * (double)__uint_as_float(ctrl->haar_max_bits));
    ctrl->sigma_max = sig1;
    ctrl->lambdas_set = 1;
  }
  __syncthreads();
  const double lamL = (double)ctrl->lambda_L;
  const bool has_sigma = a.persist->has_sigma != 0;
  if (tid < n) {
    const int i = tid;
    int r = 0;
    for (int j = 0; j < n; ++j)
      r += (sh.lam[j] > sh.lam[i]) || (sh.lam[j] == sh.lam[i] && j < i);
    sh.rank[i] = r;
    const double s = sqrt(fmax(sh.lam[i], 0.0));
    const double s1 = fmax(s - lamL, 0.0);
    double s2 = has_sigma ? s1 - a.lambda_p * (s1 - a.sigma_prev[r]) : s1;
    if (s <= a.rank_tau * sig1) s2 = 0.0;
    sh.f[i] = s > 0.0 ? s2 / s : 0.0;
    a.sigma_out[r] = s2;
  }
  __syncthreads();
  if (tid == 0) {
    double nuc = 0.0;
    int rk = 0;
    for (int r = 0; r < n; ++r) {
      const double s2 = a.sigma_out[r];
      nuc += s2;
      rk += s2 > 0.0;
    }
    ctrl->nuclear_cur = nuc;
    ctrl->rank_cur = rk;
    ctrl->v_valid = 1;
  }
  // 5. W = V diag(f) V^H and the eigenvectors for the next warm start
  for (int e = tid; e < n * n; e += kEigThreads) {
    const int i = e / n, j = e - (e / n) * n;
    float2 s = make_float2(0.f, 0.f);
    for (int k = 0; k < n; ++k) {
      const float fk = (float)sh.f[k];
      if (fk != 0.f) s = cadd(s, cscale(cmul(sh.V[i * kLd + k], cconj(sh.V[j * kLd + k])), fk));
    }
    a.W[i * n + j] = s;
    a.V[i * n + j] = sh.V[i * kLd + j];
  }
}

cudaError_t launch_eig(const EigArgs& a, cudaStream_t st) {
  const size_t smem = sizeof(EigShared) + (a.eig_fp64 ? sizeof(EigShared64) : 0);
  static size_t set_for = 0;
  if (smem > 48 * 1024 && set_for < smem) {
    cudaError_t e = cudaFuncSetAttribute(k_eig, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(sizeof(EigShared) + sizeof(EigShared64)));
    if (e != cudaSuccess) return e;
    set_for = sizeof(EigShared) + sizeof(EigShared64);
  }
  k_eig<<<1, kEigThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace lps
