// Serving loop for real-time recursive reconstruction of many concurrent sessions.
//
// Not in the paper, which reconstructs one sequence. A session is one recursive plan (its
// coil maps, L, S, prior support and singular values stay resident on the device between
// frames) with its own CUDA stream. Sessions are admitted against a device-memory budget
// (lps_estimate_device_bytes of each). Frames are submitted as they arrive; a frame leaves
// the server's queue for the device as soon as fewer than `max_inflight` frames are on the
// device (continuous batching: it does not wait for other frames to finish), behind the
// earlier frames of its own session (the recursion of Sec. 3 is sequential in t) and
// concurrently with the other sessions' frames. A frame is done when its result L + S is in
// the session's output buffer; its latency runs from the arrival time given at submission to
// that point, on one clock shared by the host and the device (a reference event recorded when
// the server was created).
#include "plan_internal.h"

#include <chrono>
#include <deque>
#include <map>
#include <memory>
#include <vector>

using namespace lps;

namespace lps {
cudaError_t launch_combine(const float2* L, const float2* S, float2* out, long long n, cudaStream_t st);
}

namespace {

struct Session {
  lps_plan* plan = nullptr;
  cudaStream_t st = nullptr;
  float2* out = nullptr;      // L + S of the last completed frame
  size_t bytes = 0;           // admitted device bytes
  int queued = 0;             // frames submitted and not yet completed
  bool shared = false;        // the server's single stream
  bool tuned = false;         // launch shapes picked (autotune on the first frame)
};

struct Frame {
  long long ticket;
  int session;
  std::vector<uint8_t> mask;
  const void* kdata;          // caller-owned until the frame is done
  double arrival;
  cudaEvent_t done = nullptr;
  bool issued = false, finished = false;
  double latency = 0.0, completion = 0.0;
};

}  // namespace

struct lps_server {
  lps_server_config cfg{};
  size_t used = 0;
  std::map<int, Session> sessions;
  int next_session = 1;
  long long next_ticket = 1;
  std::deque<long long> pending;                    // submitted, not yet on the device
  std::map<long long, std::unique_ptr<Frame>> frames;
  int inflight = 0;
  cudaStream_t ref_st = nullptr;
  cudaStream_t shared_st = nullptr;   // single_stream: the one stream of every session
  cudaEvent_t ref = nullptr;
  std::chrono::steady_clock::time_point t0;
};

namespace {

double host_now(const lps_server* S) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - S->t0).count();
}

// Issue one frame on its session's stream: mask, data, the frame graph, L + S, done event.
int issue(lps_server* S, Frame& f) {
  Session& s = S->sessions.at(f.session);
  lps_plan* P = s.plan;
  int nl = 0;
  int rc = lps_set_mask(P, f.mask.data(), &nl);
  if (rc) return rc;
  if ((rc = lps_set_data(P, f.kdata, nl))) return rc;
  if (S->cfg.autotune && !s.tuned) {
    if ((rc = lps_autotune(P, nullptr))) return rc;
    s.tuned = true;
  }
  if ((rc = lps_reconstruct_frame(P, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr))) return rc;
  if (launch_combine(P->L, P->S, s.out, P->g.N, s.st) != cudaSuccess) {
    set_err("launch of the L + S kernel failed");
    return LPS_ERR_CUDA;
  }
  CK(cudaEventCreateWithFlags(&f.done, cudaEventDefault));
  CK(cudaEventRecord(f.done, s.st));
  f.issued = true;
  ++S->inflight;
  return LPS_OK;
}

// Retire finished frames and move queued ones to the device while slots are free.
int progress(lps_server* S) {
  for (auto& kv : S->frames) {
    Frame& f = *kv.second;
    if (!f.issued || f.finished) continue;
    const cudaError_t q = cudaEventQuery(f.done);
    if (q == cudaErrorNotReady) continue;
    CK(q);
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, S->ref, f.done));
    f.completion = ms * 1e-3;
    f.latency = f.completion - f.arrival;
    f.finished = true;
    --S->inflight;
    --S->sessions.at(f.session).queued;
  }
  while (!S->pending.empty() && (S->cfg.max_inflight <= 0 || S->inflight < S->cfg.max_inflight)) {
    Frame& f = *S->frames.at(S->pending.front());
    S->pending.pop_front();
    const int rc = issue(S, f);
    if (rc) return rc;
  }
  return LPS_OK;
}

int close_session(lps_server* S, int id) {
  auto it = S->sessions.find(id);
  if (it == S->sessions.end()) return LPS_ERR_INVALID_ARG;
  Session& s = it->second;
  if (s.st) cudaStreamSynchronize(s.st);
  lps_plan_destroy(s.plan);
  if (s.out) cudaFree(s.out);
  if (s.st && !s.shared) cudaStreamDestroy(s.st);
  S->used -= s.bytes;
  S->sessions.erase(it);
  return LPS_OK;
}

}  // namespace

extern "C" {

int lps_server_create(const lps_server_config* cfg, lps_server** out) {
  ARG(cfg != nullptr && out != nullptr, "NULL argument");
  ARG(cfg->hbm_budget_bytes > 0 && cfg->max_inflight >= 0, "bad server config");
  for (int r : cfg->reserved) ARG(r == 0, "reserved fields must be zero");
  ARG(cfg->single_stream == 0 || cfg->single_stream == 1, "single_stream must be 0 or 1");
  ARG(cfg->autotune == 0 || cfg->autotune == 1, "autotune must be 0 or 1");
  lps_server* S = new lps_server();
  S->cfg = *cfg;
  if (cudaStreamCreateWithFlags(&S->ref_st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&S->ref) != cudaSuccess || cudaEventRecord(S->ref, S->ref_st) != cudaSuccess ||
      cudaEventSynchronize(S->ref) != cudaSuccess) {
    set_err("server clock setup failed");
    delete S;
    return LPS_ERR_CUDA;
  }
  if (cfg->single_stream && cudaStreamCreateWithFlags(&S->shared_st, cudaStreamNonBlocking) != cudaSuccess) {
    set_err("stream creation failed");
    cudaEventDestroy(S->ref);
    cudaStreamDestroy(S->ref_st);
    delete S;
    return LPS_ERR_CUDA;
  }
  S->t0 = std::chrono::steady_clock::now();
  *out = S;
  return LPS_OK;
}

int lps_server_destroy(lps_server* S) {
  if (!S) return LPS_OK;
  std::vector<int> ids;
  for (auto& kv : S->sessions) ids.push_back(kv.first);
  for (int id : ids) close_session(S, id);
  for (auto& kv : S->frames)
    if (kv.second->done) cudaEventDestroy(kv.second->done);
  if (S->ref) cudaEventDestroy(S->ref);
  if (S->ref_st) cudaStreamDestroy(S->ref_st);
  if (S->shared_st) cudaStreamDestroy(S->shared_st);
  delete S;
  return LPS_OK;
}

double lps_server_now(lps_server* S) { return S ? host_now(S) : 0.0; }

int lps_server_open(lps_server* S, const lps_params* p, const void* coils, int* session) {
  ARG(S != nullptr && p != nullptr && coils != nullptr && session != nullptr, "NULL argument");
  ARG(p->recursive == 1, "server sessions are recursive (params.recursive = 1)");
  size_t need = 0;
  int rc = lps_estimate_device_bytes(p, &need);
  if (rc) return rc;
  if (S->used + need > S->cfg.hbm_budget_bytes) {
    set_err("session needs %zu bytes; %zu of %zu in use", need, S->used, S->cfg.hbm_budget_bytes);
    return LPS_ERR_ADMISSION;
  }
  Session s;
  if (S->shared_st) {
    s.st = S->shared_st;
    s.shared = true;
  } else {
    CK(cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking));
  }
  auto drop_stream = [&] {
    if (!s.shared) cudaStreamDestroy(s.st);
  };
  if ((rc = lps_plan_create(p, s.st, &s.plan))) {
    drop_stream();
    return rc;
  }
  const size_t img = (size_t)p->nx * p->ny * p->nz * sizeof(float2);
  if (cudaMalloc(&s.out, img) != cudaSuccess) {
    lps_plan_destroy(s.plan);
    drop_stream();
    set_err("output buffer allocation failed");
    return LPS_ERR_OOM;
  }
  if ((rc = lps_set_coils(s.plan, coils))) {
    lps_plan_destroy(s.plan);
    cudaFree(s.out);
    drop_stream();
    return rc;
  }
  s.bytes = need;
  S->used += need;
  const int id = S->next_session++;
  S->sessions[id] = s;
  *session = id;
  return LPS_OK;
}

int lps_server_close(lps_server* S, int session) {
  ARG(S != nullptr, "server is NULL");
  auto it = S->sessions.find(session);
  ARG(it != S->sessions.end(), "unknown session %d", session);
  ARG(it->second.queued == 0, "session %d has frames in flight", session);
  return close_session(S, session);
}

int lps_server_plan(lps_server* S, int session, lps_plan** out) {
  ARG(S != nullptr && out != nullptr, "NULL argument");
  auto it = S->sessions.find(session);
  ARG(it != S->sessions.end(), "unknown session %d", session);
  *out = it->second.plan;
  return LPS_OK;
}

size_t lps_server_bytes_in_use(lps_server* S) { return S ? S->used : 0; }

int lps_server_submit(lps_server* S, int session, const uint8_t* mask, const void* kdata, double arrival,
                      long long* ticket) {
  ARG(S != nullptr && mask != nullptr && kdata != nullptr && ticket != nullptr, "NULL argument");
  auto it = S->sessions.find(session);
  ARG(it != S->sessions.end(), "unknown session %d", session);
  const Geom& g = it->second.plan->g;
  auto f = std::make_unique<Frame>();
  f->ticket = S->next_ticket++;
  f->session = session;
  f->mask.assign(mask, mask + (size_t)g.ny * g.nz);
  f->kdata = kdata;
  f->arrival = arrival;
  *ticket = f->ticket;
  ++it->second.queued;
  S->pending.push_back(f->ticket);
  S->frames[f->ticket] = std::move(f);
  return progress(S);
}

int lps_server_poll(lps_server* S, long long ticket, double* latency, double* completion) {
  ARG(S != nullptr, "server is NULL");
  int rc = progress(S);
  if (rc) return rc;
  auto it = S->frames.find(ticket);
  ARG(it != S->frames.end(), "unknown ticket %lld", ticket);
  if (!it->second->finished) return 0;
  if (latency) *latency = it->second->latency;
  if (completion) *completion = it->second->completion;
  return 1;
}

int lps_server_wait(lps_server* S, long long ticket, double* latency, double* completion) {
  ARG(S != nullptr, "server is NULL");
  for (;;) {
    int rc = lps_server_poll(S, ticket, latency, completion);
    if (rc != 0) return rc < 0 ? rc : LPS_OK;
    auto it = S->frames.find(ticket);
    if (it->second->issued) {
      CK(cudaEventSynchronize(it->second->done));
    } else {
      // queued behind full slots: wait for the oldest frame on the device
      for (auto& kv : S->frames)
        if (kv.second->issued && !kv.second->finished) {
          CK(cudaEventSynchronize(kv.second->done));
          break;
        }
    }
  }
}

int lps_server_release(lps_server* S, long long ticket) {
  ARG(S != nullptr, "server is NULL");
  auto it = S->frames.find(ticket);
  ARG(it != S->frames.end(), "unknown ticket %lld", ticket);
  ARG(it->second->finished, "frame %lld is not done", ticket);
  if (it->second->done) cudaEventDestroy(it->second->done);
  S->frames.erase(it);
  return LPS_OK;
}

int lps_server_result(lps_server* S, int session, void* out) {
  ARG(S != nullptr && out != nullptr, "NULL argument");
  auto it = S->sessions.find(session);
  ARG(it != S->sessions.end(), "unknown session %d", session);
  Session& s = it->second;
  const size_t img = (size_t)s.plan->g.N * sizeof(float2);
  CK(cudaMemcpyAsync(out, s.out, img, cudaMemcpyDefault, s.st));
  CK(cudaStreamSynchronize(s.st));
  return LPS_OK;
}

}  // extern "C"
