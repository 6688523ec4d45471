// Host side of the C ABI declared in include/lps_api.h: plan lifetime, validation, device
// buffers, the per-frame launch sequence of Algorithm 1 (Sec. 3) and its CUDA graph.
#include "plan_internal.h"

#include <cmath>
#include <cstddef>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

using namespace lps;

namespace lps {
cudaError_t launch_gram_plane(const float2* X, const float2* S, const Geom& g, float2* gram_part, int nparts,
                              cudaStream_t st);
cudaError_t launch_combine(const float2* L, const float2* S, float2* out, long long n, cudaStream_t st);
}  // namespace lps

namespace lps {

thread_local char g_err[512] = "";

void set_err(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

}  // namespace lps

namespace lps {

// The slab's share of the reduction record of x-slab sharding, summed in a fixed order: the
// Gram partials (entry by entry over the partials), the data-consistency statistics and the
// sparse step's (a warp each, lanes then shuffles), and max |T(X_0)| from the control block.
__global__ void __launch_bounds__(256) k_slab_pack(const float2* __restrict__ gram_part, int nparts, int nc,
                                                   const float* __restrict__ dc_part, int ndc,
                                                   const float* __restrict__ lrs_part, int nlrs,
                                                   const DevCtrl* __restrict__ ctrl, float* __restrict__ rec) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  float2* G = reinterpret_cast<float2*>(rec + kSlabRecHead);
  const int nn = nc * nc;
  for (int e = tid; e < nn; e += blockDim.x) {
    float2 acc = make_float2(0.f, 0.f);
    for (int q = 0; q < nparts; ++q) acc = cadd(acc, gram_part[(long long)q * nn + e]);
    G[e] = acc;
  }
  if (w == 0) {
    float r2 = 0.f, d2 = 0.f, o2 = 0.f;
    for (int i = lane; i < ndc; i += 32) {
      const float4 q = reinterpret_cast<const float4*>(dc_part)[i];
      r2 += q.x;
      d2 += q.y;
      o2 += q.z;
    }
    for (int o = 16; o > 0; o >>= 1) {
      r2 += __shfl_xor_sync(0xffffffffu, r2, o);
      d2 += __shfl_xor_sync(0xffffffffu, d2, o);
      o2 += __shfl_xor_sync(0xffffffffu, o2, o);
    }
    if (lane == 0) {
      rec[0] = r2;
      rec[1] = d2;
      rec[2] = o2;
      rec[3] = 0.f;
    }
  } else if (w == 1) {
    float l1 = 0.f, cnt = 0.f;
    for (int i = lane; i < nlrs; i += 32) {
      l1 += lrs_part[2 * i];
      cnt += lrs_part[2 * i + 1];
    }
    for (int o = 16; o > 0; o >>= 1) {
      l1 += __shfl_xor_sync(0xffffffffu, l1, o);
      cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if (lane == 0) {
      rec[4] = l1;
      rec[5] = cnt;
      rec[6] = rec[7] = 0.f;
    }
  } else if (tid == 64) {
    rec[kSlabRecHead + 2 * nn] = __uint_as_float(ctrl->haar_max_bits);
  }
}

cudaError_t launch_slab_pack(const float2* gram_part, int nparts, int nc, const float* dc_part, int ndc,
                             const float* lrs_part, int nlrs, const DevCtrl* ctrl, float* rec, cudaStream_t st) {
  k_slab_pack<<<1, 256, 0, st>>>(gram_part, nparts, nc, dc_part, ndc, lrs_part, nlrs, ctrl, rec);
  return cudaGetLastError();
}

}  // namespace lps

namespace {

bool make_fft_plan(int n, FftPlan& p) {
  p.n = n;
  p.np = 0;
  int r = n;
  auto push = [&](int v) {
    if (p.np >= kMaxPasses) return false;
    p.r[p.np++] = v;
    return true;
  };
  while (r % 16 == 0 && r != 32 && r != 64 && r != 128 && r != 512) {
    if (!push(16)) return false;
    r /= 16;
  }
  // remaining power of two: 32 = 8x4, 64 = 8x8, 128 = 16x8, 512 = 16x16x2 handled above
  if (r % 128 == 0) {
    if (!push(16) || !push(8)) return false;
    r /= 128;
  }
  while (r % 8 == 0) {
    if (!push(8)) return false;
    r /= 8;
  }
  while (r % 4 == 0) {
    if (!push(4)) return false;
    r /= 4;
  }
  while (r % 2 == 0) {
    if (!push(2)) return false;
    r /= 2;
  }
  for (int f : {3, 5, 7}) {
    while (r % f == 0) {
      if (!push(f)) return false;
      r /= f;
    }
  }
  for (int f = 11; r > 1 && f <= 64; f += 2) {
    while (r % f == 0) {
      if (!push(f)) return false;
      r /= f;
    }
  }
  return r == 1;
}

std::vector<float2> twiddles(int n) {
  std::vector<float2> t(n);
  for (int q = 0; q < n; ++q) {
    const double ang = 2.0 * M_PI * (double)q / (double)n;
    t[q] = make_float2((float)std::cos(ang), (float)(-std::sin(ang)));
  }
  return t;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace


namespace {

template <typename T>
int dalloc(lps_plan* P, T** ptr, size_t count) {
  const size_t b = count * sizeof(T);
  CK(cudaMalloc((void**)ptr, b > 0 ? b : 16));
  P->dev_bytes += b;
  return LPS_OK;
}

// Carve `count` elements from the plan's arena (256-byte aligned).
template <typename T>
int aalloc(lps_plan* P, T** ptr, size_t count) {
  const size_t b = ((count * sizeof(T) + 255) / 256) * 256;
  if (P->arena_used + b > P->arena_bytes) {
    set_err("internal arena overflow");
    return LPS_ERR_OOM;
  }
  *ptr = reinterpret_cast<T*>(P->arena + P->arena_used);
  P->arena_used += b;
  return LPS_OK;
}

// Gram partials the eigen kernel sums: from the data-consistency epilogue in float32, from
// the tensor-core Gram kernel in the precision modes.
int gram_parts(const Geom& g, int precision) {
  return precision == LPS_FP32 ? dc_gram_parts(g) : gram_tc_parts(g);
}
int gram_part_capacity(const Geom& g) { return std::max(g.nx, gram_tc_parts(g)); }

size_t arena_size(const Geom& g, int max_iters) {
  auto r = [](size_t b) { return ((b + 255) / 256) * 256; };
  size_t s = 0;
  s += r((size_t)gram_part_capacity(g) * g.nc * g.nc * sizeof(float2));   // gram partials
  s += 4 * r((size_t)g.nc * g.nc * sizeof(float2));      // W, V, float64 mode: Gram, refined V
  s += r((size_t)g.nc * g.nc * sizeof(double2)) + r((size_t)g.nc * sizeof(double));   // A, eigenvalues
  s += r((size_t)g.nxt * sizeof(float2)) + r((size_t)g.ny * sizeof(float2)) + r((size_t)g.nz * sizeof(float2));
  s += r((size_t)g.plane * sizeof(int));                  // line table
  s += r((size_t)g.nx * 4 * sizeof(float)) + 2 * r((size_t)g.ntiles * 2 * sizeof(float));   // statistic partials
  s += 2 * r((size_t)g.nc * sizeof(double));
  s += 3 * r((size_t)(g.N / 32) * sizeof(uint32_t));   // support: prior, output, second output
  s += r(sizeof(DevPersist)) + r(sizeof(DevCtrl)) + r((size_t)(max_iters + 2) * sizeof(IterRec));
  return s;
}

int validate(const lps_params* p, Geom* gout) {
  ARG(p != nullptr, "params is NULL");
  for (int r : p->reserved) ARG(r == 0, "reserved fields must be zero");
  ARG(p->nx >= 8 && p->ny >= 8 && p->nz >= 1, "sizes must be nx, ny >= 8, nz >= 1");
  ARG(p->nx % 8 == 0 && p->ny % 8 == 0, "nx and ny must be multiples of 8");
  ARG(p->nx <= 1024 && p->ny <= 1024, "nx, ny <= 1024");
  ARG(p->ncoil >= 1 && p->ncoil <= 64, "ncoil must be in 1..64");
  ARG(p->layout == LPS_LAYOUT_SLICES || p->layout == LPS_LAYOUT_FRAMES, "layout must be SLICES or FRAMES");
  ARG(p->fft_z == 0 || p->fft_z == 1, "fft_z must be 0 or 1");
  // Casorati columns: the slices (layout "slices"), or frames of frame_slices slices each
  const int fs = p->frame_slices ? p->frame_slices : 1;
  ARG(fs >= 1 && fs <= 128, "frame_slices must be 0..128");
  ARG(p->layout == LPS_LAYOUT_FRAMES || fs == 1, "frame_slices applies to LPS_LAYOUT_FRAMES");
  ARG(p->nz % fs == 0, "nz must be a multiple of frame_slices");
  if (p->layout == LPS_LAYOUT_FRAMES && fs == 1 && p->fft_z != 0) {
    // a column is one 2D frame with its own ky lines: the per-slice 2D encode
    set_err("LPS_LAYOUT_FRAMES with 2D frames (frame_slices 1) takes fft_z = 0");
    return LPS_ERR_UNSUPPORTED;
  }
  if (fs > 1 && (p->precision != LPS_FP32 || p->nx_total != 0)) {
    set_err("3D frames (frame_slices > 1) run the float32 path on whole volumes");
    return LPS_ERR_UNSUPPORTED;
  }
  ARG(p->wavelet_levels >= 1 && p->wavelet_levels <= 3, "wavelet_levels must be 1..3");
  ARG(p->wavelet_dims == 0 || p->wavelet_dims == 2 || p->wavelet_dims == 3, "wavelet_dims must be 2 or 3");
  ARG(p->wavelet_dims != 3 || p->nz % (1 << p->wavelet_levels) == 0,
      "the 3D Haar needs nz a multiple of 2^wavelet_levels");
  ARG(p->wavelet_dims != 3 || fs == 1 || fs % (1 << p->wavelet_levels) == 0,
      "the 3D Haar of 3D frames needs frame_slices a multiple of 2^wavelet_levels");
  ARG(p->max_iters >= 1 && p->max_iters <= 4096, "max_iters must be 1..4096");
  ARG(std::isfinite(p->lambda_L_rel) && p->lambda_L_rel >= 0, "lambda_L_rel must be finite, >= 0");
  ARG(std::isfinite(p->lambda_S_rel) && p->lambda_S_rel >= 0, "lambda_S_rel must be finite, >= 0");
  ARG(p->lambda_p >= 0 && p->lambda_p <= 1, "lambda_p must be in [0, 1]");
  ARG(p->rank_tau >= 0 && p->rank_tau < 1, "rank_tau must be in [0, 1)");
  ARG(p->tol >= 0 && std::isfinite(p->tol), "tol must be finite, >= 0");
  ARG(p->precision == LPS_FP32 || p->precision == LPS_TF32_REFINE || p->precision == LPS_BF16_REFINE,
      "precision must be LPS_FP32, LPS_TF32_REFINE or LPS_BF16_REFINE");
  ARG(p->eig_precision == LPS_EIG_FP32 || p->eig_precision == LPS_EIG_FP64, "bad eig_precision");
  ARG(p->support_rule == 0 || p->support_rule == 1, "bad support_rule");
  ARG(p->recursive == 0 || p->recursive == 1, "recursive must be 0 or 1");
  ARG(p->coil_format == LPS_COILS_FP32 || p->coil_format == LPS_COILS_FP16,
      "coil_format must be LPS_COILS_FP32 or LPS_COILS_FP16");
  ARG(p->data_format == LPS_DATA_FP32 || p->data_format == LPS_DATA_FP16,
      "data_format must be LPS_DATA_FP32 or LPS_DATA_FP16");
  if (p->nz / fs > LPS_MAX_NC || p->nz > 128) {
    set_err("%d Casorati columns of %d slices: at most LPS_MAX_NC = %d columns and 128 slices", p->nz / fs, fs,
            LPS_MAX_NC);
    return LPS_ERR_UNSUPPORTED;
  }
  // x-slab of a larger volume: nx_total = 0 means the whole volume
  const int nxt = p->nx_total ? p->nx_total : p->nx;
  ARG(p->nx_total == 0 || (p->nx_total >= p->nx && p->nx_total <= 1024 && p->nx_total % 8 == 0),
      "nx_total must be 0 or a multiple of 8 in nx..1024");
  ARG(p->x0 >= 0 && p->x0 % 8 == 0 && p->x0 + p->nx <= nxt, "x0 must be a multiple of 8 with x0 + nx <= nx_total");
  Geom g{};
  g.nx = p->nx;
  g.nxt = nxt;
  g.x0 = p->x0;
  g.ny = p->ny;
  g.nz = p->nz;
  g.ncoil = p->ncoil;
  g.cs = fs;
  g.nc = p->nz / fs;
  g.zn = (fs > 1 && p->fft_z) ? fs : p->nz;
  g.plane = p->ny * p->nz;
  g.nyp = p->ny + 1;
  g.planeP = p->nz * g.nyp + ((p->nz * g.nyp) & 1);
  g.fft_z = p->fft_z;
  g.J = p->wavelet_levels;
  g.wz = p->wavelet_dims == 3 ? 1 : 0;
  g.ntiles = (p->nx / 8) * (p->ny / 8);
  g.N = (long long)p->nx * p->ny * p->nz;
  g.scale_yz = (float)(1.0 / std::sqrt((double)p->ny * (p->fft_z ? g.zn : 1)));
  g.scale_x = (float)(1.0 / std::sqrt((double)nxt));
  if (!make_fft_plan(p->ny, g.py) || !make_fft_plan(g.zn, g.pz) || !make_fft_plan(nxt, g.px)) {
    set_err("FFT lengths need prime factors <= 64 and at most %d passes", kMaxPasses);
    return LPS_ERR_UNSUPPORTED;
  }
  // runtime-sized DC kernel: with more planes than SMs, read the coil maps from global memory
  // (two CTAs per SM) when that fits; lps_autotune measures both
  if (g.nx > 152) {
    Geom gd = g;
    gd.dc_direct = 1;
    g.dc_direct = dc_smem_bytes(gd) <= 113 * 1024 ? 1 : 0;
  }
  // 128 x 16 planes: the update runs on the register-transform kernel (four coil groups; their
  // sums in shared memory when there are more than four coils)
  if (g.ny == 128 && g.nz == 16) g.dc_reg_groups = g.ncoil > 4 ? 104 : 4;
  // planes of ny = 16 Q by even nz <= 32: the update's coil loop on register transforms
  g.dc_rt = dc_rt_geometry(g) ? 1 : 0;
  if (dc_ept(g) < 0 || dc_smem_bytes(g) > 227 * 1024) {
    set_err("x-plane of %d x %d does not fit one CTA", p->ny, p->nz);
    return LPS_ERR_UNSUPPORTED;
  }
  g.mpad = 0;
  if (gout) *gout = g;
  return LPS_OK;
}

int free_plan(lps_plan* P) {
  if (!P) return LPS_OK;
  if (P->gexec) cudaGraphExecDestroy(P->gexec);
  if (P->graph) cudaGraphDestroy(P->graph);
  void* bufs[] = {P->X, P->L, P->S, P->S2, P->R, P->coils, P->dhyb, P->kstage, P->hscratch, P->istage, P->arena,
                  P->Lnew, P->coils_h, P->dhyb_h};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (P->h_ctrl) cudaFreeHost(P->h_ctrl);
  if (P->h_persist_slots) cudaFreeHost(P->h_persist_slots);
  if (P->h_lines_slots) cudaFreeHost(P->h_lines_slots);
  for (int k = 0; k < lps_plan::kSlots; ++k)
    if (P->slot_done[k]) cudaEventDestroy(P->slot_done[k]);
  if (P->cap) cudaStreamDestroy(P->cap);
  if (P->side) cudaStreamDestroy(P->side);
  if (P->cap_side) cudaStreamDestroy(P->cap_side);
  if (P->ev_fork) cudaEventDestroy(P->ev_fork);
  if (P->ev_join) cudaEventDestroy(P->ev_join);
  for (cudaEvent_t e : P->ev) cudaEventDestroy(e);
  delete P;
  return LPS_OK;
}

size_t support_words(const Geom& g) { return (size_t)(g.N / 32); }

// Next pinned staging slot, once the upload last made from it has landed.
int acquire_slot(lps_plan* P, int* slot) {
  const int k = P->slot_next;
  if (P->slot_pending[k]) {
    CK(cudaEventSynchronize(P->slot_done[k]));
    P->slot_pending[k] = false;
  }
  *slot = k;
  return LPS_OK;
}

// Marks the uploads enqueued from `slot` and moves to the next slot.
int release_slot(lps_plan* P, int slot) {
  CK(cudaEventRecord(P->slot_done[slot], P->st));
  P->slot_pending[slot] = true;
  P->slot_next = (slot + 1) % lps_plan::kSlots;
  return LPS_OK;
}

// Host-owned fields: nlines, has_sup, has_sigma; v_valid is written by the eigen kernel and
// uploaded only when the host resets or restores it. `slot` >= 0: already acquired.
int upload_persist(lps_plan* P, bool with_v = false, int slot = -1) {
  int rc;
  if (slot < 0 && (rc = acquire_slot(P, &slot))) return rc;
  DevPersist* src = P->h_persist_slots + slot;
  *src = P->hp;
  const size_t n = with_v ? sizeof(DevPersist) : offsetof(DevPersist, v_valid);
  CK(cudaMemcpyAsync(P->persist, src, n, cudaMemcpyHostToDevice, P->st));
  return release_slot(P, slot);
}

// Grow the line-dependent buffers to hold m lines.
int ensure_lines(lps_plan* P, int m) {
  if (m <= P->m_cap) return LPS_OK;
  const int cap = (m + 1) & ~1;
  CK(cudaStreamSynchronize(P->st));
  if (P->dhyb) cudaFree(P->dhyb);
  if (P->kstage) cudaFree(P->kstage);
  if (P->hscratch) cudaFree(P->hscratch);
  if (P->dhyb_h) cudaFree(P->dhyb_h);
  P->dhyb = P->kstage = P->hscratch = nullptr;
  P->dhyb_h = nullptr;
  const size_t hyb = (size_t)P->g.nx * P->g.ncoil * cap + 4;
  int rc;
  if ((rc = dalloc(P, &P->dhyb, hyb))) return rc;
  if (P->p.data_format == LPS_DATA_FP16 && (rc = dalloc(P, &P->dhyb_h, hyb))) return rc;
  if ((rc = dalloc(P, &P->kstage, (size_t)P->g.ncoil * cap * P->g.nxt + 4))) return rc;
  if ((rc = dalloc(P, &P->hscratch, hyb))) return rc;
  P->m_cap = cap;
  P->g.mpad = cap;
  P->graph_valid = false;
  return LPS_OK;
}

DcArgs dc_args(lps_plan* P) {
  DcArgs a{};
  a.g = P->g;
  a.coils = P->coils;
  a.coils_h = P->coils_h;
  a.dhyb = P->dhyb;
  a.dhyb_h = P->dhyb_h;
  a.lines = P->lines;
  a.tw_y = P->tw_y;
  a.tw_z = P->tw_z;
  a.persist = P->persist;
  return a;
}

#define LK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      set_err("launch %s failed: %s", #call, cudaGetErrorString(e_));                  \
      return LPS_ERR_CUDA;                                                            \
    }                                                                                 \
  } while (0)

// Event pair around one launch when profiling (only while building the frame graph).
int prof_begin(lps_plan* P, int cls, cudaStream_t st) {
  if (!P->profiling || (st != P->cap && st != P->cap_side)) return LPS_OK;
  const size_t need = 2 * (size_t)(P->ev_used + 1);
  while (P->ev.size() < need) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    P->ev.push_back(e);
  }
  if (P->ev_class.size() < (size_t)P->ev_used + 1) P->ev_class.resize(P->ev_used + 1);
  P->ev_class[P->ev_used] = cls;
  CK(cudaEventRecordWithFlags(P->ev[2 * P->ev_used], st, cudaEventRecordExternal));
  return LPS_OK;
}
int prof_end(lps_plan* P, cudaStream_t st) {
  if (!P->profiling || (st != P->cap && st != P->cap_side)) return LPS_OK;
  CK(cudaEventRecordWithFlags(P->ev[2 * P->ev_used + 1], st, cudaEventRecordExternal));
  ++P->ev_used;
  return LPS_OK;
}
#define PROF(cls, stmt)                                  \
  do {                                                   \
    int prc_;                                            \
    if ((prc_ = prof_begin(P, cls, st))) return prc_;    \
    stmt;                                                \
    if ((prc_ = prof_end(P, st))) return prc_;           \
  } while (0)

GramTcArgs gram_tc_args(lps_plan* P, const float2* S, bool with_ctrl = true) {
  GramTcArgs a{};
  a.g = P->g;
  a.X = P->X;
  a.S = S;
  a.gram_part = P->gram_part;
  a.ctrl = with_ctrl ? P->ctrl : nullptr;
  return a;
}

// Step (0): X_0 = E^H d, L_0 := X_0, S_0 = 0, Gram of X_0, max |T(X_0)|.
int enqueue_init(lps_plan* P, cudaStream_t st) {
  CK(cudaMemsetAsync(P->ctrl, 0, sizeof(DevCtrl), st));
  // an inactive batch member starts "converged": every kernel of the frame returns at once
  CK(cudaMemcpyAsync(&P->ctrl->converged, &P->persist->skip, sizeof(int), cudaMemcpyDeviceToDevice, st));
  // Each frame starts its eigendecomposition from scratch unless the plan reconstructs a
  // sequence, where the previous frame's eigenvectors are the warm start.
  if (!P->p.recursive) CK(cudaMemsetAsync(&P->persist->v_valid, 0, sizeof(int), st));
  const bool tc = P->p.precision != LPS_FP32;
  DcArgs a = dc_args(P);
  a.X = P->X;
  a.L_out = P->L;
  a.S_out = P->S;
  a.gram_part = tc ? nullptr : P->gram_part;
  a.ctrl = P->ctrl;
  PROF(3, LK(launch_dc(a, kDcAdjoint, st)));
  if (tc) PROF(4, LK(launch_gram_tc(gram_tc_args(P, nullptr), P->p.precision, st)));
  LrsArgs l{};
  l.g = P->g;
  l.X = P->X;
  l.L = P->L;
  l.S = P->S2;
  l.lrs_part = P->lrs_part;
  l.persist = P->persist;
  l.ctrl = P->ctrl;
  l.haar_max_only = 1;
  PROF(3, LK(launch_lrs(l, st)));
  return LPS_OK;
}

// `i`: index of the iteration within its run; the statistics of the previous iteration are in
// the sparse-step partial buffer i & 1.
EigArgs eig_args(lps_plan* P, int iter, int finalize, int i) {
  EigArgs e{};
  e.g = P->g;
  e.gram_part = P->gram_part;
  e.nparts = gram_parts(P->g, P->p.precision);
  e.dc_part = P->dc_part;
  e.ndc = P->g.nx;
  e.lrs_part = (i & 1) ? P->lrs_part2 : P->lrs_part;
  e.lrs_parts = lrs_blocks(P->g);
  if (P->slab_rec) {
    // x-slab sharding: the Gram and the statistics come reduced over all slabs in one record
    e.gram_part = reinterpret_cast<const float2*>(P->slab_rec + kSlabRecHead);
    e.nparts = 1;
    e.dc_part = P->slab_rec;
    e.ndc = 1;
    e.lrs_part = P->slab_rec + 4;
    e.lrs_parts = 1;
  }
  e.W = P->W;
  e.V = P->V;
  e.sigma_prev = P->sigma_prev;
  e.sigma_out = P->sigma_out;
  e.hist = P->hist;
  e.persist = P->persist;
  e.ctrl = P->ctrl;
  e.lambda_L_rel = P->p.lambda_L_rel;
  e.lambda_S_rel = P->p.lambda_S_rel;
  e.lambda_p = P->p.lambda_p;
  e.rank_tau = P->p.rank_tau;
  e.tol = P->p.tol;
  e.lambda_p_f = (float)P->p.lambda_p;
  e.rank_tau_f = (float)P->p.rank_tau;
  e.tol_f = (float)P->p.tol;
  e.iter = iter;
  e.finalize = finalize;
  e.eig_fp64 = P->p.eig_precision == LPS_EIG_FP64;
  return e;
}

// Iteration k of Algorithm 1. The sparse step (3) needs only X_{k-1} and L_{k-1}, so it runs
// on a second stream beside the eigendecomposition of steps (1)-(2); the data-consistency
// kernel of step (4) joins both, forms L_k = (X_{k-1} - S_{k-1}) W in its prologue (or takes
// the tensor-core reprojection) and writes X_k, L_k and the next Gram:
//   main:  eig_k [-> reproj_tc_k] ----------+-> DC_k [-> gram_tc_k]
//   side:  (after DC_{k-1}) sparse_k -------+
// The sparse step's outputs (S, support words, statistic partials) alternate between two
// buffers: the i-th iteration of a run reads S_{k-1} from buffer i & 1 and writes iteration k
// to buffer (i + 1) & 1, so the eigen kernel, which runs beside the next sparse step, still
// reads the previous iteration's partials; enqueue_settle moves the last completed
// iteration's buffers into place at the end of the run.
int enqueue_iter(lps_plan* P, int k, int i, cudaStream_t st, cudaStream_t side) {
  const bool tc = P->p.precision != LPS_FP32;
  float2* Sprev = (i & 1) ? P->S2 : P->S;
  float2* Snew = (i & 1) ? P->S : P->S2;
  CK(cudaEventRecord(P->ev_fork, st));
  CK(cudaStreamWaitEvent(side, P->ev_fork, 0));
  LrsArgs l{};
  l.g = P->g;
  l.X = P->X;
  l.L = P->L;
  l.S = Snew;
  l.sup_prior = P->sup_prior;
  l.sup_out = (i & 1) ? P->sup_out : P->sup_out2;
  l.lrs_part = (i & 1) ? P->lrs_part : P->lrs_part2;
  l.persist = P->persist;
  l.ctrl = P->ctrl;
  l.lambda_S_rel = P->p.lambda_S_rel;
  l.support_rule = P->p.support_rule;
  {
    int prc;
    if ((prc = prof_begin(P, 1, side))) return prc;
    LK(launch_lrs(l, side));
    if ((prc = prof_end(P, side))) return prc;
  }
  CK(cudaEventRecord(P->ev_join, side));
  if (P->p.eig_precision == LPS_EIG_FP64) {
    // float32 Jacobi, float64 Rayleigh-Ritz refinement over nc CTAs, then the SVT steps
    EigArgs e1 = eig_args(P, k, 0, i);
    e1.part = 1;
    e1.Gout = P->G64in;
    e1.lam64 = P->lam64;
    PROF(2, LK(launch_eig(e1, st)));
    RitzArgs ra{};
    ra.n = P->g.nc;
    ra.G = P->G64in;
    ra.V = P->V;
    ra.A = P->A64;
    ra.Vout = P->Vref;
    ra.lam64 = P->lam64;
    ra.ctrl = P->ctrl;
    PROF(2, LK(launch_ritz64(ra, st)));
    EigArgs e2 = eig_args(P, k, 0, i);
    e2.part = 2;
    e2.lam64 = P->lam64;
    e2.Vin = P->Vref;
    PROF(2, LK(launch_eig(e2, st)));
  } else {
    PROF(2, LK(launch_eig(eig_args(P, k, 0, i), st)));
  }
  if (tc) {
    ReprojTcArgs r{};
    r.g = P->g;
    r.X = P->X;
    r.S = Sprev;
    r.W = P->W;
    r.Lnew = P->Lnew;
    r.ctrl = P->ctrl;
    PROF(5, LK(launch_reproj_tc(r, P->p.precision, st)));
  }
  CK(cudaStreamWaitEvent(st, P->ev_join, 0));
  DcArgs a = dc_args(P);
  a.S = Snew;
  a.Sprev = Sprev;
  a.W = tc ? nullptr : P->W;
  a.Lpre = tc ? P->Lnew : nullptr;
  a.Lbuf = P->L;
  a.X = P->X;
  a.gram_part = tc ? nullptr : P->gram_part;
  a.dc_part = P->dc_part;
  a.ctrl = P->ctrl;
  PROF(0, LK(launch_dc(a, kDcUpdate, st)));
  if (tc) PROF(4, LK(launch_gram_tc(gram_tc_args(P, Snew), P->p.precision, st)));
  return LPS_OK;
}

// End of a run whose first iteration was k0: the last completed iteration (the eigen kernel
// may have stopped the run early) decides on the device which buffers hold the result.
int enqueue_settle(lps_plan* P, int k0, cudaStream_t st) {
  LK(launch_settle(P->ctrl, k0, P->S, P->S2, P->g.N, P->sup_out, P->sup_out2, (long long)support_words(P->g),
                   P->lrs_part, P->lrs_part2, 2 * lrs_blocks(P->g), st));
  return LPS_OK;
}

// Statistics of the last iteration of a run of n iterations (its partials are in buffer n & 1).
int enqueue_finalize(lps_plan* P, int k_last, int n, cudaStream_t st) {
  PROF(2, LK(launch_eig(eig_args(P, k_last + 1, 1, n), st)));
  return LPS_OK;
}

int enqueue_frame(lps_plan* P, cudaStream_t st) {
  int rc;
  if ((rc = enqueue_init(P, st))) return rc;
  cudaStream_t side = (st == P->cap) ? P->cap_side : P->side;
  for (int k = 1; k <= P->p.max_iters; ++k)
    if ((rc = enqueue_iter(P, k, k - 1, st, side))) return rc;
  if ((rc = enqueue_finalize(P, P->p.max_iters, P->p.max_iters, st))) return rc;
  if ((rc = enqueue_settle(P, 1, st))) return rc;
  if (P->p.recursive) {
    const size_t w = support_words(P->g);
    CK(cudaMemcpyAsync(P->sup_prior, P->sup_out, w * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(P->sigma_prev, P->sigma_out, P->g.nc * sizeof(double), cudaMemcpyDeviceToDevice, st));
    // persist.has_sup / has_sigma: nonzero byte pattern
    CK(cudaMemsetAsync(&P->persist->has_sup, 1, 2 * sizeof(int), st));
  }
  return LPS_OK;
}

int build_graph(lps_plan* P) {
  if (P->graph_valid) return LPS_OK;
  if (P->gexec) {
    cudaGraphExecDestroy(P->gexec);
    P->gexec = nullptr;
  }
  P->ev_used = 0;
  CK(cudaStreamBeginCapture(P->cap, cudaStreamCaptureModeRelaxed));
  int rc = enqueue_frame(P, P->cap);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(P->cap, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  CK(e);
  e = cudaGraphInstantiate(&P->gexec, graph, 0);
  if (P->graph) cudaGraphDestroy(P->graph);
  P->graph = graph;
  CK(e);
  P->graph_valid = true;
  ++P->graph_gen;
  return LPS_OK;
}

int read_stats(lps_plan* P, lps_stats* s) {
  CK(cudaMemcpyAsync(P->h_ctrl, P->ctrl, sizeof(DevCtrl), cudaMemcpyDeviceToHost, P->st));
  CK(cudaStreamSynchronize(P->st));
  const DevCtrl& c = *P->h_ctrl;
  if (c.err & kErrTimeout) {
    set_err("a bounded device wait gave up");
    return LPS_ERR_TIMEOUT;
  }
  if (c.err & kErrNonfinite) {
    set_err("non-finite residual or singular values");
    return LPS_ERR_NONFINITE;
  }
  if (!s) return LPS_OK;
  std::memset(s, 0, sizeof(*s));
  s->iters = c.iters_done;
  s->lambda_L = c.lambda_L;
  s->lambda_S = c.lambda_S;
  s->sigma_max = c.sigma_max;
  if (c.iters_done >= 1) {
    IterRec r;
    CK(cudaMemcpy(&r, P->hist + (c.iters_done - 1), sizeof(IterRec), cudaMemcpyDeviceToHost));
    s->rank = r.rank;
    s->resid_norm2 = r.resid2;
    s->nuclear = r.nuclear;
    s->l1_off_support = r.l1;
    s->objective = iter_objective(r, c.lambda_L, c.lambda_S);
    s->rel_change = r.rel_change;
  }
  // support count from the last sparse-step partials
  const int nb = lrs_blocks(P->g);
  std::vector<float> part((size_t)nb * 2);
  CK(cudaMemcpy(part.data(), P->lrs_part, part.size() * sizeof(float), cudaMemcpyDeviceToHost));
  long long cnt = 0;
  for (int t = 0; t < nb; ++t) cnt += (long long)part[(size_t)t * 2 + 1];
  s->support_count = cnt;
  return LPS_OK;
}

int copy_out(lps_plan* P, void* dst, const void* src, size_t bytes, bool* host_dst) {
  if (!dst) return LPS_OK;
  CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, P->st));
  if (!is_device_ptr(dst)) *host_dst = true;
  return LPS_OK;
}

// Host bookkeeping once a frame graph has been enqueued: the state is the frame's result and,
// in recursive mode, the graph has installed the frame's support and sigma as the prior.
void frame_done(lps_plan* P) {
  P->state_ready = true;
  P->iters_done = P->p.max_iters;
  if (P->p.recursive) {
    P->hp.has_sup = 1;
    P->hp.has_sigma = 1;
  }
}

int need_ready(lps_plan* P) {
  if (!P) {
    set_err("plan is NULL");
    return LPS_ERR_INVALID_ARG;
  }
  if (!P->have_coils || !P->have_mask || !P->have_data) {
    set_err("set_coils, set_mask and set_data must precede iterations");
    return LPS_ERR_STATE;
  }
  return LPS_OK;
}

}  // namespace

namespace lps {
// Validated geometry of a parameter set (used by entry points that run without a plan).
int make_geom(const lps_params* p, Geom* g) { return validate(p, g); }
int plan_build_graph(lps_plan* P) { return build_graph(P); }
int plan_need_ready(lps_plan* P) { return need_ready(P); }
int plan_upload_persist(lps_plan* P, bool with_v) { return upload_persist(P, with_v); }
int plan_frame_done(lps_plan* P) {
  frame_done(P);
  return LPS_OK;
}
DcArgs plan_dc_args(lps_plan* P) { return dc_args(P); }
bool plan_is_device_ptr(const void* p) { return is_device_ptr(p); }
}  // namespace lps

extern "C" {

int lps_version(void) { return 1; }

const char* lps_last_error(void) { return g_err; }

const char* lps_status_string(int s) {
  switch (s) {
    case LPS_OK: return "LPS_OK";
    case LPS_ERR_INVALID_ARG: return "LPS_ERR_INVALID_ARG";
    case LPS_ERR_OOM: return "LPS_ERR_OOM";
    case LPS_ERR_CUDA: return "LPS_ERR_CUDA";
    case LPS_ERR_TIMEOUT: return "LPS_ERR_TIMEOUT";
    case LPS_ERR_NONFINITE: return "LPS_ERR_NONFINITE";
    case LPS_ERR_ADMISSION: return "LPS_ERR_ADMISSION";
    case LPS_ERR_STATE: return "LPS_ERR_STATE";
    case LPS_ERR_UNSUPPORTED: return "LPS_ERR_UNSUPPORTED";
    default: return "LPS_ERR_UNKNOWN";
  }
}

int lps_params_init(lps_params* p) {
  if (!p) return LPS_ERR_INVALID_ARG;
  std::memset(p, 0, sizeof(*p));
  p->layout = LPS_LAYOUT_SLICES;
  p->fft_z = 1;
  p->wavelet_levels = 3;
  p->wavelet_dims = 2;
  p->max_iters = 50;
  p->lambda_L_rel = 0.01;
  p->lambda_S_rel = 0.005;
  p->lambda_p = 0.5;
  p->rank_tau = 1e-3;
  p->tol = 0.0;
  p->precision = LPS_FP32;
  p->eig_precision = LPS_EIG_FP32;
  p->support_rule = LPS_SUPPORT_THRESHOLD;
  p->recursive = 0;
  return LPS_OK;
}

size_t lps_support_words(const lps_params* p) {
  if (!p) return 0;
  return (size_t)p->nx * p->ny * p->nz / 32;
}

int lps_estimate_device_bytes(const lps_params* p, size_t* bytes) {
  Geom g;
  int rc = validate(p, &g);
  if (rc) return rc;
  ARG(bytes != nullptr, "bytes is NULL");
  const size_t N = (size_t)g.N;
  const size_t m = (size_t)((g.plane / 2 + 1) & ~1);   // first frame at 50% of the lines
  size_t b = 0;
  b += 4 * N * 8;                              // X, L, S, recon
  if (p->precision != LPS_FP32) b += N * 8;    // reprojection output
  b += (size_t)g.ncoil * N * 8;                // coils
  if (p->coil_format == LPS_COILS_FP16) b += (size_t)g.ncoil * N * 4;   // half-precision copy
  if (p->data_format == LPS_DATA_FP16) b += ((size_t)g.nx * g.ncoil * m + 4) * 4;   // half samples
  b += 2 * ((size_t)g.nx * g.ncoil * m + 4) * 8 + ((size_t)g.nxt * g.ncoil * m + 4) * 8;   // hybrid, scratch, staging
  b += (size_t)gram_part_capacity(g) * g.nc * g.nc * 8 + 2 * g.nc * g.nc * 8;
  b += (size_t)g.nx * 4 + (size_t)g.ntiles * 16 + 2 * N / 8;
  b += (size_t)(p->max_iters + 2) * sizeof(IterRec) + 4096;
  *bytes = b;
  return LPS_OK;
}

int lps_plan_create(const lps_params* p, void* stream, lps_plan** out) {
  ARG(out != nullptr, "out is NULL");
  *out = nullptr;
  Geom g;
  int rc = validate(p, &g);
  if (rc) return rc;
  lps_plan* P = new lps_plan();
  P->p = *p;
  P->g = g;
  P->st = (cudaStream_t)stream;
  const size_t N = (size_t)g.N;
  auto fail = [&](int r) {
    free_plan(P);
    return r;
  };
  if ((rc = dalloc(P, &P->X, N))) return fail(rc);
  if ((rc = dalloc(P, &P->L, N))) return fail(rc);
  if ((rc = dalloc(P, &P->S, N))) return fail(rc);
  if ((rc = dalloc(P, &P->S2, N))) return fail(rc);
  if ((rc = dalloc(P, &P->R, N))) return fail(rc);
  if ((rc = dalloc(P, &P->istage, N))) return fail(rc);
  if ((rc = dalloc(P, &P->coils, N * g.ncoil))) return fail(rc);
  if (p->coil_format == LPS_COILS_FP16 && (rc = dalloc(P, &P->coils_h, N * g.ncoil))) return fail(rc);
  if (p->precision != LPS_FP32 && (rc = dalloc(P, &P->Lnew, N))) return fail(rc);
  P->arena_bytes = arena_size(g, p->max_iters);
  if ((rc = dalloc(P, &P->arena, P->arena_bytes))) return fail(rc);
  if ((rc = aalloc(P, &P->ctrl, 1))) return fail(rc);
  if ((rc = aalloc(P, &P->persist, 1))) return fail(rc);
  if ((rc = aalloc(P, &P->W, (size_t)g.nc * g.nc))) return fail(rc);
  if ((rc = aalloc(P, &P->V, (size_t)g.nc * g.nc))) return fail(rc);
  if ((rc = aalloc(P, &P->G64in, (size_t)g.nc * g.nc))) return fail(rc);
  if ((rc = aalloc(P, &P->Vref, (size_t)g.nc * g.nc))) return fail(rc);
  if ((rc = aalloc(P, &P->A64, (size_t)g.nc * g.nc))) return fail(rc);
  if ((rc = aalloc(P, &P->lam64, (size_t)g.nc))) return fail(rc);
  if ((rc = aalloc(P, &P->sigma_out, (size_t)g.nc))) return fail(rc);
  if ((rc = aalloc(P, &P->sigma_prev, (size_t)g.nc))) return fail(rc);
  if ((rc = aalloc(P, &P->dc_part, (size_t)g.nx * 4))) return fail(rc);
  if ((rc = aalloc(P, &P->lrs_part, (size_t)g.ntiles * 2))) return fail(rc);
  if ((rc = aalloc(P, &P->lrs_part2, (size_t)g.ntiles * 2))) return fail(rc);
  if ((rc = aalloc(P, &P->tw_x, (size_t)g.nxt))) return fail(rc);
  if ((rc = aalloc(P, &P->tw_y, (size_t)g.ny))) return fail(rc);
  if ((rc = aalloc(P, &P->tw_z, (size_t)g.nz))) return fail(rc);
  if ((rc = aalloc(P, &P->lines, (size_t)g.plane))) return fail(rc);
  if ((rc = aalloc(P, &P->hist, (size_t)p->max_iters + 2))) return fail(rc);
  if ((rc = aalloc(P, &P->gram_part, (size_t)gram_part_capacity(g) * g.nc * g.nc))) return fail(rc);
  if ((rc = aalloc(P, &P->sup_out, support_words(g)))) return fail(rc);
  if ((rc = aalloc(P, &P->sup_out2, support_words(g)))) return fail(rc);
  if ((rc = aalloc(P, &P->sup_prior, support_words(g)))) return fail(rc);
  if (cudaMallocHost((void**)&P->h_ctrl, sizeof(DevCtrl)) != cudaSuccess ||
      cudaMallocHost((void**)&P->h_persist_slots, lps_plan::kSlots * sizeof(DevPersist)) != cudaSuccess ||
      cudaMallocHost((void**)&P->h_lines_slots, (size_t)lps_plan::kSlots * g.plane * sizeof(int)) != cudaSuccess) {
    set_err("pinned host allocation failed");
    return fail(LPS_ERR_OOM);
  }
  std::memset(&P->hp, 0, sizeof(DevPersist));
  if (cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&P->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&P->cap_side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    set_err("stream creation failed");
    return fail(LPS_ERR_CUDA);
  }
  for (int k = 0; k < lps_plan::kSlots; ++k)
    if (cudaEventCreateWithFlags(&P->slot_done[k], cudaEventDisableTiming) != cudaSuccess) {
      set_err("event creation failed");
      return fail(LPS_ERR_CUDA);
    }
  auto up = [&](float2* d, int n) -> int {
    std::vector<float2> t = twiddles(n);
    CK(cudaMemcpy(d, t.data(), n * sizeof(float2), cudaMemcpyHostToDevice));
    return LPS_OK;
  };
  if ((rc = up(P->tw_x, g.nxt)) || (rc = up(P->tw_y, g.ny)) || (rc = up(P->tw_z, g.zn))) return fail(rc);
  if (cudaMemset(P->persist, 0, sizeof(DevPersist)) != cudaSuccess ||
      cudaMemset(P->ctrl, 0, sizeof(DevCtrl)) != cudaSuccess ||
      cudaMemset(P->dc_part, 0, g.nx * 4 * sizeof(float)) != cudaSuccess ||
      cudaMemset(P->lrs_part, 0, g.ntiles * 2 * sizeof(float)) != cudaSuccess ||
      cudaMemset(P->lrs_part2, 0, g.ntiles * 2 * sizeof(float)) != cudaSuccess ||
      cudaMemset(P->sup_prior, 0, support_words(g) * 4) != cudaSuccess ||
      cudaMemset(P->sup_out, 0, support_words(g) * 4) != cudaSuccess ||
      cudaMemset(P->sup_out2, 0, support_words(g) * 4) != cudaSuccess) {
    set_err("device memset failed");
    return fail(LPS_ERR_CUDA);
  }
  *out = P;
  return LPS_OK;
}

int lps_plan_destroy(lps_plan* P) {
  if (!P) return LPS_OK;
  if (P->st) cudaStreamSynchronize(P->st);
  return free_plan(P);
}

int lps_set_stream(lps_plan* P, void* stream) {
  ARG(P != nullptr, "plan is NULL");
  P->st = (cudaStream_t)stream;
  return LPS_OK;
}

int lps_plan_device_bytes(const lps_plan* P, size_t* bytes) {
  ARG(P != nullptr && bytes != nullptr, "NULL argument");
  *bytes = P->dev_bytes;
  return LPS_OK;
}

int lps_set_coils(lps_plan* P, const void* coils) {
  ARG(P != nullptr && coils != nullptr, "NULL argument");
  CK(cudaMemcpyAsync(P->coils, coils, (size_t)P->g.N * P->g.ncoil * sizeof(float2), cudaMemcpyDefault,
                     P->st));
  if (P->coils_h) LK(launch_round_half(P->coils, P->coils_h, (long long)P->g.N * P->g.ncoil, P->st));
  P->have_coils = true;
  return LPS_OK;
}

int lps_set_mask(lps_plan* P, const uint8_t* mask, int* nlines) {
  ARG(P != nullptr && mask != nullptr, "NULL argument");
  const int ny = P->g.ny, nz = P->g.nz;
  std::vector<uint8_t> hbuf;
  const uint8_t* h = mask;
  if (is_device_ptr(mask)) {
    hbuf.resize((size_t)ny * nz);
    CK(cudaMemcpyAsync(hbuf.data(), mask, hbuf.size(), cudaMemcpyDeviceToHost, P->st));
    CK(cudaStreamSynchronize(P->st));
    h = hbuf.data();
  }
  int m = 0;
  for (size_t i = 0; i < (size_t)ny * nz; ++i) m += h[i] != 0;
  ARG(m > 0, "mask has no sampled entry");
  int rc = ensure_lines(P, m);
  if (rc) return rc;
  int slot;
  if ((rc = acquire_slot(P, &slot))) return rc;
  int* hl = P->h_lines_slots + (size_t)slot * P->g.plane;
  int k = 0;
  for (int a = 0; a < nz; ++a)
    for (int ky = 0; ky < ny; ++ky)
      if (h[(size_t)a * ny + ky]) hl[k++] = a * P->g.nyp + ky;
  CK(cudaMemcpyAsync(P->lines, hl, (size_t)m * sizeof(int), cudaMemcpyHostToDevice, P->st));
  P->nlines = m;
  P->hp.nlines = m;
  if ((rc = upload_persist(P, false, slot))) return rc;
  P->have_mask = true;
  P->have_data = false;
  P->state_ready = false;
  if (nlines) *nlines = m;
  return LPS_OK;
}

int lps_set_data(lps_plan* P, const void* kdata, int nlines) {
  ARG(P != nullptr && kdata != nullptr, "NULL argument");
  if (!P->have_mask) {
    set_err("set_mask must precede set_data");
    return LPS_ERR_STATE;
  }
  ARG(nlines == P->nlines, "nlines %d does not match the mask (%d lines)", nlines, P->nlines);
  const void* src = kdata;
  if (!is_device_ptr(kdata)) {
    CK(cudaMemcpyAsync(P->kstage, kdata, (size_t)P->g.ncoil * nlines * P->g.nxt * sizeof(float2),
                       cudaMemcpyDefault, P->st));
    src = P->kstage;
  }
  XfftArgs a{};
  a.g = P->g;
  a.in = (const float2*)src;
  a.out = P->dhyb;
  a.tw_x = P->tw_x;
  a.persist = P->persist;
  a.inverse = 1;
  LK(launch_xfft(a, P->st));
  // LPS_DATA_FP16: round the hybrid samples in place and keep the half-pair copy
  if (P->dhyb_h)
    LK(launch_round_half(P->dhyb, P->dhyb_h, (long long)P->g.nx * P->g.ncoil * P->g.mpad, P->st));
  P->have_data = true;
  P->state_ready = false;
  return LPS_OK;
}

int lps_set_prior(lps_plan* P, const uint32_t* support, const double* sigma_prev) {
  ARG(P != nullptr, "plan is NULL");
  if (support)
    CK(cudaMemcpyAsync(P->sup_prior, support, support_words(P->g) * sizeof(uint32_t), cudaMemcpyDefault,
                       P->st));
  if (sigma_prev)
    CK(cudaMemcpyAsync(P->sigma_prev, sigma_prev, P->g.nc * sizeof(double), cudaMemcpyDefault, P->st));
  P->hp.has_sup = support ? 1 : 0;
  P->hp.has_sigma = sigma_prev ? 1 : 0;
  return upload_persist(P);
}

int lps_shift_prior_columns(lps_plan* P, int shift) {
  ARG(P != nullptr, "plan is NULL");
  ARG(shift >= 1 && shift < P->g.nc, "shift must be in 1..columns-1");
  ARG(!P->g.wz, "the 3D Haar mixes the columns of a z block: its support has no per-column shift");
  // support words of one Casorati column (the coefficients of one slice or frame are
  // contiguous: the column index is the outermost of the tile-major numbering)
  const size_t wpc = (size_t)P->g.cs * P->g.nx * P->g.ny / 32;
  const size_t keep = (size_t)(P->g.nc - shift) * wpc;
  // through the second support buffer, free between frames (the ranges overlap)
  CK(cudaMemcpyAsync(P->sup_out2, P->sup_prior + shift * wpc, keep * sizeof(uint32_t), cudaMemcpyDeviceToDevice,
                     P->st));
  CK(cudaMemcpyAsync(P->sup_prior, P->sup_out2, keep * sizeof(uint32_t), cudaMemcpyDeviceToDevice, P->st));
  for (int z = P->g.nc - shift; z < P->g.nc; ++z)
    CK(cudaMemcpyAsync(P->sup_prior + z * wpc, P->sup_out2 + keep - wpc, wpc * sizeof(uint32_t),
                       cudaMemcpyDeviceToDevice, P->st));
  return LPS_OK;
}

int lps_clear_prior(lps_plan* P) {
  ARG(P != nullptr, "plan is NULL");
  P->hp.v_valid = 0;
  P->hp.has_sup = 0;
  P->hp.has_sigma = 0;
  return upload_persist(P, true);
}

int lps_iterate(lps_plan* P, int n_iters, lps_stats* stats) {
  int rc = need_ready(P);
  if (rc) return rc;
  if (P->g.nxt != P->g.nx) {
    set_err("a plan that holds a slab of the volume iterates through lps_slab_begin/iterate/end");
    return LPS_ERR_STATE;
  }
  const int done = P->state_ready ? P->iters_done : 0;
  ARG(n_iters >= 0 && done + n_iters <= P->p.max_iters, "n_iters out of range (done %d, max_iters %d)", done,
      P->p.max_iters);
  if (!P->state_ready) {
    if ((rc = enqueue_init(P, P->st))) return rc;
    P->iters_done = 0;
    P->state_ready = true;
  }
  const int k0 = P->iters_done + 1;
  for (int i = 0; i < n_iters; ++i) {
    ++P->iters_done;
    if ((rc = enqueue_iter(P, P->iters_done, i, P->st, P->side))) return rc;
  }
  if (P->iters_done > 0 && (rc = enqueue_finalize(P, P->iters_done, n_iters, P->st))) return rc;
  if ((rc = enqueue_settle(P, k0, P->st))) return rc;
  return read_stats(P, stats);
}

int lps_reconstruct_frame(lps_plan* P, void* out_recon, void* out_L, void* out_S, uint32_t* out_support,
                          double* out_sigma, lps_stats* stats) {
  int rc = need_ready(P);
  if (rc) return rc;
  if (P->g.nxt != P->g.nx) {
    set_err("a plan that holds a slab of the volume reconstructs through lps_slab_begin/iterate/end");
    return LPS_ERR_STATE;
  }
  if ((rc = build_graph(P))) return rc;
  if (P->hp.skip) {   // left over from a batch in which this plan sat out a step
    P->hp.skip = 0;
    if ((rc = upload_persist(P))) return rc;
  }
  CK(cudaGraphLaunch(P->gexec, P->st));
  frame_done(P);
  const size_t img = (size_t)P->g.N * sizeof(float2);
  bool host = false;
  if (out_recon) {
    float2* dst = is_device_ptr(out_recon) ? (float2*)out_recon : P->R;
    LK(launch_combine(P->L, P->S, dst, P->g.N, P->st));
    if (dst == P->R && (rc = copy_out(P, out_recon, P->R, img, &host))) return rc;
  }
  if ((rc = copy_out(P, out_L, P->L, img, &host))) return rc;
  if ((rc = copy_out(P, out_S, P->S, img, &host))) return rc;
  if ((rc = copy_out(P, out_support, P->sup_out, support_words(P->g) * 4, &host))) return rc;
  if ((rc = copy_out(P, out_sigma, P->sigma_out, P->g.nc * sizeof(double), &host))) return rc;
  if (stats) {
    if ((rc = read_stats(P, stats))) return rc;
    P->iters_done = stats->iters;
  } else if (host) {
    CK(cudaStreamSynchronize(P->st));
  }
  return LPS_OK;
}


int lps_set_profiling(lps_plan* P, int on) {
  ARG(P != nullptr, "plan is NULL");
  if ((on != 0) != P->profiling) {
    P->profiling = on != 0;
    P->graph_valid = false;
  }
  return LPS_OK;
}

int lps_get_kernel_times(lps_plan* P, lps_kernel_times* out) {
  ARG(P != nullptr && out != nullptr, "NULL argument");
  std::memset(out, 0, sizeof(*out));
  if (!P->profiling || !P->graph_valid) return LPS_OK;
  CK(cudaStreamSynchronize(P->st));
  for (int i = 0; i < P->ev_used; ++i) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, P->ev[2 * i], P->ev[2 * i + 1]));
    out->launches[P->ev_class[i]] += 1;
    out->ms[P->ev_class[i]] += ms;
  }
  return LPS_OK;
}

int lps_get_history(lps_plan* P, lps_iter_record* out, int max, int* count) {
  ARG(P != nullptr && out != nullptr && count != nullptr && max >= 0, "bad argument");
  CK(cudaMemcpyAsync(P->h_ctrl, P->ctrl, sizeof(DevCtrl), cudaMemcpyDeviceToHost, P->st));
  CK(cudaStreamSynchronize(P->st));
  const int n = std::min(max, P->h_ctrl->iters_done);
  std::vector<IterRec> r(n > 0 ? n : 1);
  if (n > 0) CK(cudaMemcpy(r.data(), P->hist, n * sizeof(IterRec), cudaMemcpyDeviceToHost));
  for (int i = 0; i < n; ++i) {
    out[i].resid_norm2 = r[i].resid2;
    out[i].nuclear = r[i].nuclear;
    out[i].l1_off_support = r[i].l1;
    out[i].objective = iter_objective(r[i], P->h_ctrl->lambda_L, P->h_ctrl->lambda_S);
    out[i].rel_change = r[i].rel_change;
    out[i].rank = r[i].rank;
    out[i].eig_sweeps = r[i].sweeps;
  }
  *count = n;
  return LPS_OK;
}

int lps_get_state(lps_plan* P, void* X, void* L, void* S) {
  ARG(P != nullptr, "plan is NULL");
  const size_t img = (size_t)P->g.N * sizeof(float2);
  bool host = false;
  int rc;
  if ((rc = copy_out(P, X, P->X, img, &host))) return rc;
  if ((rc = copy_out(P, L, P->L, img, &host))) return rc;
  if ((rc = copy_out(P, S, P->S, img, &host))) return rc;
  if (host) CK(cudaStreamSynchronize(P->st));
  return LPS_OK;
}

int lps_get_support(lps_plan* P, uint32_t* support, double* sigma) {
  ARG(P != nullptr, "plan is NULL");
  bool host = false;
  int rc;
  if ((rc = copy_out(P, support, P->sup_out, support_words(P->g) * 4, &host))) return rc;
  if ((rc = copy_out(P, sigma, P->sigma_out, P->g.nc * sizeof(double), &host))) return rc;
  if (host) CK(cudaStreamSynchronize(P->st));
  return LPS_OK;
}

int lps_set_state(lps_plan* P, const void* X, const void* S, const void* L_prev, double lambda_L,
                  double lambda_S, int iters_done) {
  ARG(P != nullptr && X != nullptr && S != nullptr, "NULL argument");
  ARG(iters_done >= 0 && iters_done < P->p.max_iters, "iters_done out of range");
  ARG(std::isfinite(lambda_L) && lambda_L >= 0 && std::isfinite(lambda_S) && lambda_S >= 0, "bad lambdas");
  if (!P->have_coils || !P->have_mask || !P->have_data) {
    set_err("set_coils, set_mask and set_data must precede set_state");
    return LPS_ERR_STATE;
  }
  const size_t img = (size_t)P->g.N * sizeof(float2);
  CK(cudaMemcpyAsync(P->X, X, img, cudaMemcpyDefault, P->st));
  CK(cudaMemcpyAsync(P->S, S, img, cudaMemcpyDefault, P->st));
  CK(cudaMemcpyAsync(P->L, L_prev ? L_prev : X, img, cudaMemcpyDefault, P->st));
  CK(cudaMemsetAsync(P->ctrl, 0, sizeof(DevCtrl), P->st));
  CK(cudaMemsetAsync(P->dc_part, 0, P->g.nx * 4 * sizeof(float), P->st));
  CK(cudaMemsetAsync(P->lrs_part, 0, P->g.ntiles * 2 * sizeof(float), P->st));
  DevCtrl c{};
  c.lambda_L = (float)lambda_L;
  c.lambda_S = (float)lambda_S;
  c.lambdas_set = 1;
  c.sigma_max = 0.0;
  *P->h_ctrl = c;
  CK(cudaMemcpyAsync(P->ctrl, P->h_ctrl, sizeof(DevCtrl), cudaMemcpyHostToDevice, P->st));
  if (P->p.precision != LPS_FP32)
    LK(launch_gram_tc(gram_tc_args(P, P->S, false), P->p.precision, P->st));
  else
    LK(launch_gram_plane(P->X, P->S, P->g, P->gram_part, dc_gram_parts(P->g), P->st));
  CK(cudaStreamSynchronize(P->st));
  P->state_ready = true;
  P->iters_done = iters_done;
  return LPS_OK;
}

int lps_casorati_gram(lps_plan* P, const void* X, const void* S, void* G) {
  ARG(P != nullptr && X != nullptr && G != nullptr, "NULL argument");
  ARG(is_device_ptr(X) && is_device_ptr(G) && (S == nullptr || is_device_ptr(S)), "X, S, G must be device pointers");
  int nparts;
  if (P->p.precision != LPS_FP32) {
    GramTcArgs a{};
    a.g = P->g;
    a.X = (const float2*)X;
    a.S = (const float2*)S;
    a.gram_part = P->gram_part;
    LK(launch_gram_tc(a, P->p.precision, P->st));
    nparts = gram_tc_parts(P->g);
  } else {
    nparts = P->g.nx;
    LK(launch_gram_plane((const float2*)X, (const float2*)S, P->g, P->gram_part, nparts, P->st));
  }
  LK(launch_gram_sum(P->gram_part, nparts, P->g.nc, (float2*)G, P->st));
  return LPS_OK;
}

int lps_lowrank_reproject(lps_plan* P, const void* X, const void* S, const void* W, void* L) {
  ARG(P != nullptr && X != nullptr && W != nullptr && L != nullptr, "NULL argument");
  ARG(is_device_ptr(X) && is_device_ptr(W) && is_device_ptr(L) && (S == nullptr || is_device_ptr(S)),
      "X, S, W, L must be device pointers");
  if (P->p.precision != LPS_FP32) {
    ReprojTcArgs a{};
    a.g = P->g;
    a.X = (const float2*)X;
    a.S = (const float2*)S;
    a.W = (const float2*)W;
    a.Lnew = (float2*)L;
    LK(launch_reproj_tc(a, P->p.precision, P->st));
  } else {
    LK(launch_reproj_f32((const float2*)X, (const float2*)S, (const float2*)W, (float2*)L, P->g, P->st));
  }
  return LPS_OK;
}

int lps_forward(lps_plan* P, const void* image, void* kdata) {
  ARG(P != nullptr && image != nullptr && kdata != nullptr, "NULL argument");
  if (!P->have_coils || !P->have_mask) {
    set_err("set_coils and set_mask must precede lps_forward");
    return LPS_ERR_STATE;
  }
  const size_t img = (size_t)P->g.N * sizeof(float2);
  const float2* src = (const float2*)image;
  if (!is_device_ptr(image)) {
    CK(cudaMemcpyAsync(P->istage, image, img, cudaMemcpyDefault, P->st));
    src = P->istage;
  }
  DcArgs a = dc_args(P);
  a.L = src;
  a.hyb_out = P->hscratch;
  LK(launch_dc(a, kDcForward, P->st));
  const bool dev = is_device_ptr(kdata);
  XfftArgs x{};
  x.g = P->g;
  x.in = P->hscratch;
  x.out = dev ? (float2*)kdata : P->kstage;
  x.tw_x = P->tw_x;
  x.persist = P->persist;
  x.inverse = 0;
  LK(launch_xfft(x, P->st));
  if (!dev) {
    CK(cudaMemcpyAsync(kdata, P->kstage, (size_t)P->g.ncoil * P->nlines * P->g.nxt * sizeof(float2),
                       cudaMemcpyDefault, P->st));
    CK(cudaStreamSynchronize(P->st));
  }
  return LPS_OK;
}

int lps_adjoint(lps_plan* P, const void* kdata, void* image) {
  ARG(P != nullptr && image != nullptr && kdata != nullptr, "NULL argument");
  if (!P->have_coils || !P->have_mask) {
    set_err("set_coils and set_mask must precede lps_adjoint");
    return LPS_ERR_STATE;
  }
  const float2* src = (const float2*)kdata;
  if (!is_device_ptr(kdata)) {
    CK(cudaMemcpyAsync(P->kstage, kdata, (size_t)P->g.ncoil * P->nlines * P->g.nxt * sizeof(float2),
                       cudaMemcpyDefault, P->st));
    src = P->kstage;
  }
  XfftArgs x{};
  x.g = P->g;
  x.in = src;
  x.out = P->hscratch;
  x.tw_x = P->tw_x;
  x.persist = P->persist;
  x.inverse = 1;
  LK(launch_xfft(x, P->st));
  const bool dev = is_device_ptr(image);
  DcArgs a = dc_args(P);
  a.dhyb = P->hscratch;
  a.dhyb_h = nullptr;   // the operator's own samples, in float32
  a.X = dev ? (float2*)image : P->istage;
  LK(launch_dc(a, kDcAdjoint, P->st));
  if (!dev) {
    CK(cudaMemcpyAsync(image, P->istage, (size_t)P->g.N * sizeof(float2), cudaMemcpyDefault, P->st));
    CK(cudaStreamSynchronize(P->st));
  }
  return LPS_OK;
}

int lps_data_consistency(lps_plan* P, const void* Z, void* X, double* resid_norm2) {
  ARG(P != nullptr && Z != nullptr && X != nullptr, "NULL argument");
  int rc = need_ready(P);
  if (rc) return rc;
  const size_t img = (size_t)P->g.N * sizeof(float2);
  const float2* src = (const float2*)Z;
  if (!is_device_ptr(Z)) {
    CK(cudaMemcpyAsync(P->istage, Z, img, cudaMemcpyDefault, P->st));
    src = P->istage;
  }
  const bool dev = is_device_ptr(X);
  float2* dst = dev ? (float2*)X : P->R;
  DcArgs a = dc_args(P);
  a.L = src;
  a.S = nullptr;
  a.X = dst;
  a.dc_part = P->dc_part;
  const int stall = P->stall_polls;
  P->stall_polls = 0;
  if (stall) {
    a.stall_polls = stall;
    a.err_word = &P->ctrl->err;
    CK(cudaMemsetAsync(&P->ctrl->err, 0, sizeof(int), P->st));
  }
  LK(launch_dc(a, kDcUpdate, P->st));
  if (stall) {
    int err = 0;
    CK(cudaMemcpyAsync(&err, &P->ctrl->err, sizeof(int), cudaMemcpyDeviceToHost, P->st));
    CK(cudaStreamSynchronize(P->st));
    CK(cudaMemsetAsync(&P->ctrl->err, 0, sizeof(int), P->st));
    P->state_ready = false;
    if (err & kErrTimeout) {
      set_err("data consistency: a bounded wait ran out (test hook)");
      return LPS_ERR_TIMEOUT;
    }
  }
  if (!dev) CK(cudaMemcpyAsync(X, P->R, img, cudaMemcpyDefault, P->st));
  if (resid_norm2) {
    std::vector<float> part((size_t)P->g.nx * 4);
    CK(cudaMemcpyAsync(part.data(), P->dc_part, part.size() * sizeof(float), cudaMemcpyDeviceToHost, P->st));
    CK(cudaStreamSynchronize(P->st));
    double s = 0;
    for (int i = 0; i < P->g.nx; ++i) s += part[(size_t)i * 4];
    *resid_norm2 = s;
  } else if (!dev) {
    CK(cudaStreamSynchronize(P->st));
  }
  P->state_ready = false;
  return LPS_OK;
}

int lps_test_stall_wait(lps_plan* P, int polls) {
  ARG(P != nullptr, "plan is NULL");
  ARG(polls >= 1 && polls <= (1 << 20), "polls must be in 1..2^20");
  if (!(P->g.dc_generic && !P->g.dc_direct)) {
    set_err("the stall hook needs the staged-coil runtime-sized kernel (lps_apply_tune dc_variant 1)");
    return LPS_ERR_STATE;
  }
  P->stall_polls = polls;
  return LPS_OK;
}

int lps_slab_reduction_size(const lps_plan* P, size_t* sum_floats, size_t* max_floats) {
  ARG(P != nullptr && sum_floats != nullptr && max_floats != nullptr, "NULL argument");
  *sum_floats = slab_sum_floats(P->g.nc);
  *max_floats = 1;
  return LPS_OK;
}

int lps_slab_begin(lps_plan* P, float* rec) {
  int rc = need_ready(P);
  if (rc) return rc;
  ARG(rec != nullptr && is_device_ptr(rec), "rec must be a device buffer");
  P->slab_rec = nullptr;
  if ((rc = enqueue_init(P, P->st))) return rc;
  LK(launch_slab_pack(P->gram_part, gram_parts(P->g, P->p.precision), P->g.nc, P->dc_part, P->g.nx, P->lrs_part,
                      lrs_blocks(P->g), P->ctrl, rec, P->st));
  P->iters_done = 0;
  P->state_ready = true;
  P->slab_open = true;
  return LPS_OK;
}

int lps_slab_iterate(lps_plan* P, float* rec, int k) {
  ARG(P != nullptr && rec != nullptr, "NULL argument");
  if (!P->slab_open) {
    set_err("lps_slab_begin must precede lps_slab_iterate");
    return LPS_ERR_STATE;
  }
  ARG(k == P->iters_done + 1 && k <= P->p.max_iters, "iteration %d out of order (done %d, max_iters %d)", k,
      P->iters_done, P->p.max_iters);
  if (k == 1) {
    // the maximum over the slabs of |T(X_0)| fixes lambda_S at the first iteration
    CK(cudaMemcpyAsync(&P->ctrl->haar_max_bits, rec + slab_sum_floats(P->g.nc), sizeof(float),
                       cudaMemcpyDeviceToDevice, P->st));
  }
  P->slab_rec = rec;
  const int i = k - 1;
  int rc = enqueue_iter(P, k, i, P->st, P->side);
  P->slab_rec = nullptr;
  if (rc) return rc;
  // the sparse step of iteration k wrote its partials to buffer (i + 1) & 1
  LK(launch_slab_pack(P->gram_part, gram_parts(P->g, P->p.precision), P->g.nc, P->dc_part, P->g.nx,
                      (i & 1) ? P->lrs_part : P->lrs_part2, lrs_blocks(P->g), P->ctrl, rec, P->st));
  P->iters_done = k;
  return LPS_OK;
}

int lps_slab_end(lps_plan* P, const float* rec, lps_stats* stats) {
  ARG(P != nullptr && rec != nullptr, "NULL argument");
  if (!P->slab_open || P->iters_done < 1) {
    set_err("lps_slab_end needs lps_slab_begin and at least one lps_slab_iterate");
    return LPS_ERR_STATE;
  }
  const int K = P->iters_done;
  P->slab_rec = rec;
  int rc = enqueue_finalize(P, K, K, P->st);
  P->slab_rec = nullptr;
  if (rc) return rc;
  if ((rc = enqueue_settle(P, 1, P->st))) return rc;
  if (P->p.recursive) {
    const size_t w = support_words(P->g);
    CK(cudaMemcpyAsync(P->sup_prior, P->sup_out, w * sizeof(uint32_t), cudaMemcpyDeviceToDevice, P->st));
    CK(cudaMemcpyAsync(P->sigma_prev, P->sigma_out, P->g.nc * sizeof(double), cudaMemcpyDeviceToDevice, P->st));
    CK(cudaMemsetAsync(&P->persist->has_sup, 1, 2 * sizeof(int), P->st));
    P->hp.has_sup = 1;
    P->hp.has_sigma = 1;
  }
  P->slab_open = false;
  return read_stats(P, stats);
}

// Checkpoint layout: header, prior support words, prior sigma, L, S, X, lambdas.
struct CkptHeader {
  uint32_t magic, version;
  int nx, ny, nz, ncoil, J, has_sup, has_sigma, iters_done, v_valid, wz;   // wz + 256 * slices per column
  double lambda_L, lambda_S;
};

int lps_session_export(lps_plan* P, void* buf, size_t* bytes) {
  ARG(P != nullptr && bytes != nullptr, "NULL argument");
  const size_t w = support_words(P->g), img = (size_t)P->g.N * sizeof(float2);
  const size_t vb = (size_t)P->g.nc * P->g.nc * sizeof(float2);
  const size_t need = sizeof(CkptHeader) + w * 4 + P->g.nc * sizeof(double) + 3 * img + vb;
  if (!buf) {
    *bytes = need;
    return LPS_OK;
  }
  ARG(*bytes >= need, "buffer too small (%zu < %zu)", *bytes, need);
  CK(cudaMemcpyAsync(P->h_ctrl, P->ctrl, sizeof(DevCtrl), cudaMemcpyDeviceToHost, P->st));
  DevPersist dp;
  CK(cudaMemcpyAsync(&dp, P->persist, sizeof(DevPersist), cudaMemcpyDeviceToHost, P->st));
  CK(cudaStreamSynchronize(P->st));
  CkptHeader h{0x4c50531a, 2, P->g.nx, P->g.ny, P->g.nz, P->g.ncoil, P->g.J, dp.has_sup,
               dp.has_sigma, P->iters_done, dp.v_valid, P->g.wz + 256 * P->g.cs, P->h_ctrl->lambda_L, P->h_ctrl->lambda_S};
  unsigned char* o = (unsigned char*)buf;
  std::memcpy(o, &h, sizeof(h));
  o += sizeof(h);
  CK(cudaMemcpy(o, P->sup_prior, w * 4, cudaMemcpyDeviceToHost));
  o += w * 4;
  CK(cudaMemcpy(o, P->sigma_prev, P->g.nc * sizeof(double), cudaMemcpyDeviceToHost));
  o += P->g.nc * sizeof(double);
  CK(cudaMemcpy(o, P->L, img, cudaMemcpyDeviceToHost));
  o += img;
  CK(cudaMemcpy(o, P->S, img, cudaMemcpyDeviceToHost));
  o += img;
  CK(cudaMemcpy(o, P->X, img, cudaMemcpyDeviceToHost));
  o += img;
  CK(cudaMemcpy(o, P->V, vb, cudaMemcpyDeviceToHost));
  *bytes = need;
  return LPS_OK;
}

int lps_session_import(lps_plan* P, const void* buf, size_t bytes) {
  ARG(P != nullptr && buf != nullptr, "NULL argument");
  const size_t w = support_words(P->g), img = (size_t)P->g.N * sizeof(float2);
  const size_t vb = (size_t)P->g.nc * P->g.nc * sizeof(float2);
  const size_t need = sizeof(CkptHeader) + w * 4 + P->g.nc * sizeof(double) + 3 * img + vb;
  ARG(bytes >= need, "checkpoint too small");
  CkptHeader h;
  std::memcpy(&h, buf, sizeof(h));
  ARG(h.magic == 0x4c50531a && h.version == 2, "not a checkpoint of this library");
  ARG(h.nx == P->g.nx && h.ny == P->g.ny && h.nz == P->g.nz && h.J == P->g.J && h.wz == P->g.wz + 256 * P->g.cs,
      "checkpoint shape mismatch");
  const unsigned char* i = (const unsigned char*)buf + sizeof(h);
  CK(cudaStreamSynchronize(P->st));
  CK(cudaMemcpy(P->sup_prior, i, w * 4, cudaMemcpyHostToDevice));
  i += w * 4;
  CK(cudaMemcpy(P->sigma_prev, i, P->g.nc * sizeof(double), cudaMemcpyHostToDevice));
  i += P->g.nc * sizeof(double);
  CK(cudaMemcpy(P->L, i, img, cudaMemcpyHostToDevice));
  i += img;
  CK(cudaMemcpy(P->S, i, img, cudaMemcpyHostToDevice));
  i += img;
  CK(cudaMemcpy(P->X, i, img, cudaMemcpyHostToDevice));
  i += img;
  CK(cudaMemcpy(P->V, i, vb, cudaMemcpyHostToDevice));
  P->hp.has_sup = h.has_sup;
  P->hp.has_sigma = h.has_sigma;
  P->hp.v_valid = h.v_valid;
  return upload_persist(P, true);
}

}  // extern "C"
