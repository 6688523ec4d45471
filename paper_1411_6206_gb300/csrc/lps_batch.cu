// Batches of independent problems and the autotuner of the per-problem launch shapes.
//
// A batch owns one plan per problem (sizes, slice counts and coil counts may differ). Its
// frame step is one CUDA graph: every member's captured per-frame graph (step (0), the
// iterations of Algorithm 1, the recursion hand-over of Sec. 3) is a parallel branch, so one
// graph launch reconstructs one frame of every member and the branches share the GPU. A
// member without a frame to do this step is marked inactive: its graph starts with its
// control block "converged" and every kernel of the branch returns at once, so the graph
// need not be rebuilt when members finish their sequences at different times.
//
// The autotuner times, on a plan's own resident data, the candidate launch shapes of the two
// per-iteration kernels whose shape is a free choice: the data-consistency kernel (the
// compile-time plane kernel where one exists, else the runtime-sized kernel with every
// candidate ordering of FFT radix passes along y and z, with the coil planes staged in shared
// memory or read from global memory) and the sparse-step kernel (8x8 tiles per CTA). The
// fastest is installed in the plan; results are cached per geometry.
#include "plan_internal.h"

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

using namespace lps;

namespace lps {
cudaError_t launch_combine(const float2* L, const float2* S, float2* out, long long n, cudaStream_t st);
}

namespace {

// ---- FFT pass orderings ---------------------------------------------------------------

// Ordered radix sequences for a length-n transform: the power-of-two part as every ordered
// split into radices 16, 8, 4 and 2, with the odd factors (3, 5, 7, then larger primes, in
// that order) after or before it. Sorted by pass count; at most `cap` are returned, none
// with more than one pass beyond the fewest.
std::vector<FftPlan> fft_candidates(int n, int cap) {
  int a = 0, odd = n;
  while (odd % 2 == 0) {
    odd /= 2;
    ++a;
  }
  std::vector<int> oddr;
  for (int f : {3, 5, 7}) {
    while (odd % f == 0) {
      oddr.push_back(f);
      odd /= f;
    }
  }
  for (int f = 11; odd > 1 && f <= 64; f += 2) {
    while (odd % f == 0) {
      oddr.push_back(f);
      odd /= f;
    }
  }
  if (odd > 1) return {};
  std::vector<std::vector<int>> twos;
  std::vector<int> cur;
  auto rec = [&](auto&& self, int left) -> void {
    if ((int)(cur.size() + oddr.size()) > kMaxPasses) return;
    if (left == 0) {
      twos.push_back(cur);
      return;
    }
    for (int e : {4, 3, 2, 1}) {
      if (e > left) continue;
      cur.push_back(1 << e);
      self(self, left - e);
      cur.pop_back();
    }
  };
  rec(rec, a);
  std::vector<std::vector<int>> seqs;
  for (const auto& t : twos) {
    std::vector<int> s1 = t;
    s1.insert(s1.end(), oddr.begin(), oddr.end());
    seqs.push_back(s1);
    if (!oddr.empty() && !t.empty()) {
      std::vector<int> s2 = oddr;
      s2.insert(s2.end(), t.begin(), t.end());
      seqs.push_back(s2);
    }
  }
  if (seqs.empty()) return {};
  std::stable_sort(seqs.begin(), seqs.end(), [](const auto& x, const auto& y) { return x.size() < y.size(); });
  const size_t fewest = seqs.front().size();
  std::vector<FftPlan> out;
  for (const auto& s : seqs) {
    if (s.size() > fewest + 1 || (int)out.size() >= cap) break;
    FftPlan p{};
    p.n = n;
    p.np = (int)s.size();
    for (int i = 0; i < p.np; ++i) p.r[i] = s[i];
    out.push_back(p);
  }
  return out;
}

struct TuneKey {
  int nx, ny, nz, ncoil, fft_z, precision;
  bool operator<(const TuneKey& o) const {
    return std::tie(nx, ny, nz, ncoil, fft_z, precision) < std::tie(o.nx, o.ny, o.nz, o.ncoil, o.fft_z, o.precision);
  }
};
struct TuneEntry {
  lps_tune_result res;
  FftPlan py, pz;
};
std::mutex g_tune_mutex;
std::map<TuneKey, TuneEntry> g_tune_cache;

// dc_reg_groups value of a register-transform variant (3: four coil groups, their sums in
// shared memory when there are more coils than groups; 4: eight groups), 0 otherwise.
int reg_groups_of(int variant, int ncoil) {
  if (variant == 3) return ncoil > 4 ? 104 : 4;
  if (variant == 4) return 8;
  return 0;
}

void install(lps_plan* P, const TuneEntry& t) {
  const bool runtime = t.res.dc_variant == 1 || t.res.dc_variant == 2;
  P->g.dc_generic = runtime;
  P->g.dc_direct = t.res.dc_variant == 2;
  P->g.dc_reg_groups = reg_groups_of(t.res.dc_variant, P->g.ncoil);
  P->g.dc_rt = t.res.dc_variant == 5;
  if (runtime) {
    P->g.py = t.py;
    P->g.pz = t.pz;
  }
  P->g.lrs_tpc = t.res.lrs_tiles;
  P->graph_valid = false;
}

// Mean device time of `reps` launches of `fn` on the plan's stream (after one warm-up).
template <typename F>
int time_launches(lps_plan* P, cudaEvent_t e0, cudaEvent_t e1, int reps, F fn, double* us) {
  if (fn() != cudaSuccess) return LPS_ERR_CUDA;
  CK(cudaEventRecord(e0, P->st));
  for (int i = 0; i < reps; ++i)
    if (fn() != cudaSuccess) return LPS_ERR_CUDA;
  CK(cudaEventRecord(e1, P->st));
  CK(cudaEventSynchronize(e1));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  *us = 1e3 * ms / reps;
  return LPS_OK;
}

}  // namespace

// ---- batches -----------------------------------------------------------------------------

struct lps_batch {
  std::vector<lps_plan*> plans;
  std::vector<int> active;
  cudaStream_t st = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<unsigned> gens;   // member graph generations the batch graph was built from
  std::vector<int> members;     // plans in the batch graph
};

namespace {

int batch_free(lps_batch* B) {
  if (!B) return LPS_OK;
  if (B->st) cudaStreamSynchronize(B->st);
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  for (lps_plan* P : B->plans) lps_plan_destroy(P);
  delete B;
  return LPS_OK;
}

// (Re)build the batch graph when a member's frame graph was captured again.
int batch_graph(lps_batch* B) {
  std::vector<int> members;
  for (int i = 0; i < (int)B->plans.size(); ++i)
    if (B->plans[i]->graph_valid && B->plans[i]->graph) members.push_back(i);
  bool stale = B->exec == nullptr || members != B->members;
  for (size_t k = 0; !stale && k < members.size(); ++k)
    stale = B->gens[k] != B->plans[members[k]]->graph_gen;
  if (!stale) return LPS_OK;
  if (B->exec) {
    cudaGraphExecDestroy(B->exec);
    B->exec = nullptr;
  }
  if (B->graph) {
    cudaGraphDestroy(B->graph);
    B->graph = nullptr;
  }
  CK(cudaGraphCreate(&B->graph, 0));
  B->gens.clear();
  for (int i : members) {
    cudaGraphNode_t node;
    CK(cudaGraphAddChildGraphNode(&node, B->graph, nullptr, 0, B->plans[i]->graph));
    B->gens.push_back(B->plans[i]->graph_gen);
  }
  CK(cudaGraphInstantiate(&B->exec, B->graph, 0));
  B->members = members;
  return LPS_OK;
}

}  // namespace

extern "C" {

int lps_autotune(lps_plan* P, lps_tune_result* out) {
  ARG(P != nullptr, "plan is NULL");
  int rc = plan_need_ready(P);
  if (rc) return rc;
  const TuneKey key{P->g.nx, P->g.ny, P->g.nz, P->g.ncoil, P->g.fft_z + 2 * P->g.cs, P->p.precision};
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      install(P, it->second);
      if (out) {
        *out = it->second.res;
        out->cached = 1;
      }
      return LPS_OK;
    }
  }
  // scratch control block (never converged) and events
  DevCtrl* ctrl = nullptr;
  CK(cudaMalloc(&ctrl, sizeof(DevCtrl)));
  CK(cudaMemsetAsync(ctrl, 0, sizeof(DevCtrl), P->st));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  TuneEntry best{};
  std::memset(&best.res, 0, sizeof(best.res));
  best.res.dc_us = 1e30;
  best.res.lrs_us = 1e30;
  const Geom g0 = P->g;
  const bool fp32 = P->p.precision == LPS_FP32;
  int count = 0;
  auto dc_time = [&](const Geom& g, double* us) {
    DcArgs a = plan_dc_args(P);
    a.g = g;
    a.L = P->istage;    // scratch input and output: the plan's state is left alone
    a.S = nullptr;
    a.X = P->R;
    a.gram_part = fp32 ? P->gram_part : nullptr;
    a.ctrl = ctrl;
    return time_launches(P, e0, e1, 5, [&] { return launch_dc(a, kDcUpdate, P->st); }, us);
  };
  // data-consistency kernel: the compile-time plane kernel, the register-transform kernel in
  // both group counts where the plane has one, the register-transform coil loop of k_dc, then
  // the runtime-sized candidates
  if (dc_rt_geometry(g0) && !P->coils_h) {
    Geom g = g0;
    g.dc_generic = 0;
    g.dc_reg_groups = 0;
    g.dc_rt = 1;
    if (dc_rt_applies(g)) {
      double us;
      if ((rc = dc_time(g, &us))) goto done;
      ++count;
      if (us < best.res.dc_us) {
        best.res.dc_variant = 5;
        best.res.dc_us = us;
      }
    }
  }
  if (dc_has_fixed(g0)) {
    for (int variant : {0, 3, 4}) {
      Geom g = g0;
      g.dc_generic = 0;
      g.dc_rt = 0;
      g.dc_reg_groups = reg_groups_of(variant, g.ncoil);
      if (variant != 0 && !dc_reg_applies(g)) continue;
      double us;
      if ((rc = dc_time(g, &us))) goto done;
      ++count;
      if (us < best.res.dc_us) {
        best.res.dc_variant = variant;
        best.res.dc_us = us;
      }
    }
  }
  {
    const std::vector<FftPlan> cy = fft_candidates(g0.ny, 6);
    const std::vector<FftPlan> cz = fft_candidates(g0.zn, 4);
    for (int direct = 0; direct < 2; ++direct)
      for (const FftPlan& py : cy)
        for (const FftPlan& pz : cz) {
          Geom g = g0;
          g.dc_generic = 1;
          g.dc_direct = direct;
          g.dc_reg_groups = 0;
          g.dc_rt = 0;
          g.py = py;
          g.pz = pz;
          double us;
          if ((rc = dc_time(g, &us))) goto done;
          ++count;
          if (us < best.res.dc_us) {
            best.res.dc_us = us;
            best.res.dc_variant = 1 + direct;
            best.py = py;
            best.pz = pz;
          }
        }
  }
  // low-rank / sparse kernel: 8x8 tiles per CTA
  {
    const int tmax = std::max(1, 32 / g0.nz);
    int last = -1;
    for (int t : {tmax, tmax / 2, tmax / 4, 1}) {
      if (t < 1 || t == last) continue;
      last = t;
      Geom g = g0;
      g.lrs_tpc = t;
      LrsArgs l{};
      l.g = g;
      l.X = P->X;
      l.L = P->istage;
      l.S = P->R;
      l.sup_prior = P->sup_prior;
      l.lrs_part = P->lrs_part;
      l.persist = P->persist;
      l.ctrl = ctrl;
      double us;
      if ((rc = time_launches(P, e0, e1, 5, [&] { return launch_lrs(l, P->st); }, &us))) goto done;
      ++count;
      if (us < best.res.lrs_us) {
        best.res.lrs_us = us;
        best.res.lrs_tiles = t;
      }
    }
  }
  best.res.candidates = count;
  for (int i = 0; i < 8; ++i) {
    const bool runtime = best.res.dc_variant == 1 || best.res.dc_variant == 2;
    best.res.radix_y[i] = (runtime && i < best.py.np) ? best.py.r[i] : 0;
    best.res.radix_z[i] = (runtime && i < best.pz.np) ? best.pz.r[i] : 0;
  }
  install(P, best);
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = best;
  }
  if (out) *out = best.res;
done:
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(P->st);
  cudaFree(ctrl);
  return rc;
}

int lps_apply_tune(lps_plan* P, const lps_tune_result* t) {
  ARG(P != nullptr && t != nullptr, "NULL argument");
  ARG(t->dc_variant >= 0 && t->dc_variant <= 5, "dc_variant must be 0..5");
  ARG(t->lrs_tiles >= 1 && t->lrs_tiles <= std::max(1, 32 / P->g.nz), "lrs_tiles must be in 1..max(1, 32/nz)");
  TuneEntry e{};
  e.res = *t;
  if (t->dc_variant == 5) {
    ARG(dc_rt_geometry(P->g), "no register-transform coil loop for this plane size");
  } else if (t->dc_variant == 0 || t->dc_variant >= 3) {
    Geom g = P->g;
    g.dc_generic = 0;
    g.dc_reg_groups = reg_groups_of(t->dc_variant, g.ncoil);
    ARG(dc_has_fixed(g), "no compile-time kernel for this plane size");
    ARG(t->dc_variant == 0 || dc_reg_applies(g), "no register-transform kernel for this plane size");
  } else {
    auto plan_of = [&](const int* r, int n, FftPlan& f) -> bool {
      f = FftPlan{};
      f.n = n;
      long long prod = 1;
      for (int i = 0; i < 8 && r[i]; ++i) {
        if (r[i] < 2 || r[i] > 64) return false;
        f.r[f.np++] = r[i];
        prod *= r[i];
      }
      return f.np > 0 && prod == n;
    };
    ARG(plan_of(t->radix_y, P->g.ny, e.py), "radix_y does not factor ny");
    ARG(plan_of(t->radix_z, P->g.zn, e.pz), "radix_z does not factor the z transform length");
  }
  ARG(cudaStreamSynchronize(P->st) == cudaSuccess, "stream error");
  install(P, e);
  if (dc_smem_bytes(P->g) > 227 * 1024) {
    set_err("the plane does not fit one CTA with this variant");
    return LPS_ERR_UNSUPPORTED;
  }
  return LPS_OK;
}

int lps_autotune_clear_cache(void) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tune_cache.clear();
  return LPS_OK;
}

int lps_get_recon(lps_plan* P, void* out) {
  ARG(P != nullptr && out != nullptr, "NULL argument");
  if (!P->state_ready) {
    set_err("no reconstructed frame yet");
    return LPS_ERR_STATE;
  }
  cudaPointerAttributes at;
  const bool dev = cudaPointerGetAttributes(&at, out) == cudaSuccess &&
                   (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
  cudaGetLastError();
  float2* dst = dev ? (float2*)out : P->R;
  if (launch_combine(P->L, P->S, dst, P->g.N, P->st) != cudaSuccess) {
    set_err("launch of the L + S kernel failed");
    return LPS_ERR_CUDA;
  }
  if (!dev) {
    CK(cudaMemcpyAsync(out, P->R, (size_t)P->g.N * sizeof(float2), cudaMemcpyDeviceToHost, P->st));
    CK(cudaStreamSynchronize(P->st));
  }
  return LPS_OK;
}

int lps_batch_create(const lps_params* params, int n, void* stream, lps_batch** out) {
  ARG(out != nullptr && params != nullptr && n >= 1 && n <= 4096, "bad batch arguments");
  *out = nullptr;
  lps_batch* B = new lps_batch();
  B->st = (cudaStream_t)stream;
  for (int i = 0; i < n; ++i) {
    lps_plan* P = nullptr;
    const int rc = lps_plan_create(&params[i], stream, &P);
    if (rc) {
      batch_free(B);
      return rc;
    }
    B->plans.push_back(P);
    B->active.push_back(1);
  }
  *out = B;
  return LPS_OK;
}

int lps_batch_destroy(lps_batch* B) { return batch_free(B); }

int lps_batch_size(lps_batch* B) { return B ? (int)B->plans.size() : 0; }

int lps_batch_plan(lps_batch* B, int i, lps_plan** out) {
  ARG(B != nullptr && out != nullptr && i >= 0 && i < (int)B->plans.size(), "bad batch member");
  *out = B->plans[i];
  return LPS_OK;
}

int lps_batch_set_active(lps_batch* B, int i, int active) {
  ARG(B != nullptr && i >= 0 && i < (int)B->plans.size(), "bad batch member");
  B->active[i] = active ? 1 : 0;
  return LPS_OK;
}

int lps_batch_autotune(lps_batch* B) {
  ARG(B != nullptr, "batch is NULL");
  for (int i = 0; i < (int)B->plans.size(); ++i) {
    if (!B->active[i]) continue;
    const int rc = lps_autotune(B->plans[i], nullptr);
    if (rc) return rc;
  }
  return LPS_OK;
}

int lps_batch_reconstruct(lps_batch* B) {
  ARG(B != nullptr, "batch is NULL");
  int rc;
  int nact = 0;
  for (int i = 0; i < (int)B->plans.size(); ++i) {
    lps_plan* P = B->plans[i];
    if (!B->active[i]) continue;
    ++nact;
    if ((rc = plan_need_ready(P))) return rc;
    P->profiling = false;
    if ((rc = plan_build_graph(P))) return rc;
  }
  if (nact == 0) return LPS_OK;
  if ((rc = batch_graph(B))) return rc;
  for (int k : B->members) {
    lps_plan* P = B->plans[k];
    const int skip = B->active[k] ? 0 : 1;
    if (P->hp.skip != skip) {
      P->hp.skip = skip;
      if ((rc = plan_upload_persist(P, false))) return rc;
    }
  }
  CK(cudaGraphLaunch(B->exec, B->st));
  for (int k : B->members)
    if (B->active[k]) plan_frame_done(B->plans[k]);
  return LPS_OK;
}

int lps_batch_data_consistency(lps_batch* B, void* const* Z, void* const* X, int persistent, float* ms) {
  ARG(B != nullptr && Z != nullptr && X != nullptr, "NULL argument");
  std::vector<DcArgs> tab;
  std::vector<int> start{0};
  size_t smem = 0;
  int rc;
  for (int i = 0; i < (int)B->plans.size(); ++i) {
    if (!B->active[i]) continue;
    lps_plan* P = B->plans[i];
    if ((rc = plan_need_ready(P))) return rc;
    ARG(Z[i] != nullptr && X[i] != nullptr && plan_is_device_ptr(Z[i]) && plan_is_device_ptr(X[i]),
        "Z and X of an active member must be device pointers");
    DcArgs a = plan_dc_args(P);
    a.L = (const float2*)Z[i];
    a.S = nullptr;
    a.X = (float2*)X[i];
    a.dc_part = P->dc_part;
    if (persistent) {
      if (!dc_persist_fits(a.g)) {
        set_err("member %d: plane of %d elements does not fit the persistent form", i, a.g.plane);
        return LPS_ERR_UNSUPPORTED;
      }
      smem = std::max(smem, dc_persist_smem(a.g));
    }
    tab.push_back(a);
    start.push_back(start.back() + a.g.nx);
  }
  if (tab.empty()) return LPS_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cs = nullptr;
  DcArgs* dtab = nullptr;
  int* dint = nullptr;
  rc = LPS_OK;
  auto fail = [&](cudaError_t e) {
    set_err("%s", cudaGetErrorString(e));
    cudaGetLastError();   // a failed launch leaves nothing behind for the plans' next launches
    rc = LPS_ERR_CUDA;
  };
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) fail(e);
  if (!rc && !persistent) {
    // each member's own kernel, as parallel branches of one graph
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaGraphCreate(&graph, 0);
    for (size_t k = 0; e == cudaSuccess && k < tab.size(); ++k) {
      cudaGraph_t child = nullptr;
      e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        const cudaError_t el = launch_dc(tab[k], kDcUpdate, cs);
        e = cudaStreamEndCapture(cs, &child);
        if (e == cudaSuccess) e = el;
      }
      cudaGraphNode_t node;
      if (e == cudaSuccess) e = cudaGraphAddChildGraphNode(&node, graph, nullptr, 0, child);
      if (child) cudaGraphDestroy(child);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (e == cudaSuccess) e = cudaEventRecord(e0, B->st);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, B->st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, B->st);
    if (e != cudaSuccess) fail(e);
  } else if (!rc) {
    const int nm = (int)tab.size();
    e = cudaMalloc(&dtab, tab.size() * sizeof(DcArgs));
    if (e == cudaSuccess) e = cudaMalloc(&dint, (start.size() + 1) * sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyAsync(dtab, tab.data(), tab.size() * sizeof(DcArgs), cudaMemcpyHostToDevice, B->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dint, start.data(), start.size() * sizeof(int), cudaMemcpyHostToDevice, B->st);
    if (e == cudaSuccess) e = cudaEventRecord(e0, B->st);
    if (e == cudaSuccess) e = launch_dc_persist(dtab, dint, nm, dint + start.size(), smem, B->st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, B->st);
    if (e != cudaSuccess) fail(e);
  }
  if (!rc) {
    e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e != cudaSuccess) fail(e);
    else if (ms) *ms = t;
  }
  cudaStreamSynchronize(B->st);
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (cs) cudaStreamDestroy(cs);
  if (dtab) cudaFree(dtab);
  if (dint) cudaFree(dint);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return rc;
}

}  // extern "C"
