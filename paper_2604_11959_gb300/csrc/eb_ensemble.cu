// eb_ensemble.cu -- many independent EB instances advanced together.
//
// An ensemble holds geometry handles of any sizes (one precision, one
// device) and two state buffers per member.  One forward-Euler step of every
// member is captured once as a CUDA graph: each member's stage (bulk, near-EB
// and redistribution kernels) hangs on its own branch, forked from and
// joined to the launching stream, so the kernels of small members run side by
// side and fill the GPU.  eb_ensemble_step replays the graph (one launch per
// step, the two buffers alternating).  The autotuner times whole-ensemble
// steps over the slab height of the bulk kernel's tiles (its extent in z) and
// keeps the fastest; the states are restored afterwards.
#include "eb_handle.cuh"

#include <algorithm>
#include <vector>

using namespace ebh;

struct eb_ensemble_s {
  std::vector<eb_geom> m;
  eb_precision prec = EB_MIXED;
  int device = 0;
  std::vector<void *> buf[2];   // 5 fields per member
  int cur = 0;                  // buffer holding the current states
  std::vector<double> dt;       // time steps the graphs were captured with
  cudaGraphExec_t exec[2] = {nullptr, nullptr};   // step from buffer b to 1 - b
  std::vector<cudaStream_t> lane;
  std::vector<cudaEvent_t> ev;  // fork and join event per member
  cudaEvent_t ev_root = nullptr;
  cudaStream_t cap = nullptr;   // the graphs are captured here (the caller's stream may be the legacy one)
  size_t es = 4;

  void *field(int b, int q, int f) { return buf[b][5 * q + f]; }
  void drop_graphs() {
    for (int b = 0; b < 2; ++b)
      if (exec[b]) {
        cudaGraphExecDestroy(exec[b]);
        exec[b] = nullptr;
      }
  }
  void release() {
    drop_graphs();
    for (cudaStream_t s : lane) cudaStreamDestroy(s);
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    if (ev_root) cudaEventDestroy(ev_root);
    if (cap) cudaStreamDestroy(cap);
    for (int b = 0; b < 2; ++b)
      for (void *p : buf[b]) cudaFree(p);
    lane.clear();
    ev.clear();
    buf[0].clear();
    buf[1].clear();
  }
};

namespace {

template <typename T>
void member_stage(eb_ensemble e, int q, int from, cudaStream_t s) {
  void *src[5], *dst[5];
  for (int f = 0; f < 5; ++f) {
    src[f] = e->field(from, q, f);
    dst[f] = e->field(1 - from, q, f);
  }
  stage<T>(e->m[q], src, src, dst, e->dt[q], 0, s, false);
}

// One step of every member, buffer `from` to 1 - from, captured as a graph
// on the ensemble's own stream.
eb_status capture(eb_ensemble e, int from, cudaGraphExec_t *out) {
  cudaStream_t s = e->cap;
  cudaGraph_t graph = nullptr;
  CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "begin capture");
  cudaEventRecord(e->ev_root, s);
  for (size_t q = 0; q < e->m.size(); ++q) {
    cudaStream_t L = e->lane[q];
    cudaStreamWaitEvent(L, e->ev_root, 0);
    if (e->prec == EB_F64) member_stage<double>(e, (int)q, from, L);
    else member_stage<float>(e, (int)q, from, L);
    cudaEventRecord(e->ev[q], L);
    cudaStreamWaitEvent(s, e->ev[q], 0);
  }
  const cudaError_t ce = cudaStreamEndCapture(s, &graph);
  if (ce != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(ce, "end capture");
  }
  const cudaError_t ie = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) return cuda_fail(ie, "instantiate step graph");
  return EB_OK;
}

eb_status run_steps(eb_ensemble e, int nsteps, cudaStream_t s) {
  for (int n = 0; n < nsteps; ++n) {
    const int b = e->cur;
    if (!e->exec[b]) {
      const eb_status st = capture(e, b, &e->exec[b]);
      if (st != EB_OK) return st;
    }
    CUDA_TRY(cudaGraphLaunch(e->exec[b], s), "launch step graph");
    e->cur = 1 - b;
  }
  return EB_OK;
}

bool member_ok(eb_ensemble e, int q) { return e && q >= 0 && q < (int)e->m.size(); }

}  // namespace

extern "C" {

eb_status eb_ensemble_create(const eb_geom *members, int n, eb_ensemble *out) {
  if (!out) return fail(EB_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!members || n < 1) return fail(EB_ERR_INVALID_ARG, "members is NULL or n < 1");
  for (int q = 0; q < n; ++q)
    if (!members[q]) return fail(EB_ERR_INVALID_ARG, "a member handle is NULL");
  for (int q = 1; q < n; ++q) {
    if (members[q]->prec != members[0]->prec) return fail(EB_ERR_INVALID_ARG, "members differ in precision");
    if (members[q]->device != members[0]->device) return fail(EB_ERR_INVALID_ARG, "members are on different devices");
    for (int r = 0; r < q; ++r)
      if (members[r] == members[q]) return fail(EB_ERR_INVALID_ARG, "a handle appears twice");
  }
  int cur = -1;
  CUDA_TRY(cudaGetDevice(&cur), "current device");
  if (cur != members[0]->device) return fail(EB_ERR_INVALID_ARG, "the current device is not the members' device");
  eb_ensemble e = new eb_ensemble_s();
  e->m.assign(members, members + n);
  e->prec = members[0]->prec;
  e->device = cur;
  e->es = e->prec == EB_F64 ? sizeof(double) : sizeof(float);
  e->dt.assign(n, 0.0);
  cudaError_t err = cudaEventCreateWithFlags(&e->ev_root, cudaEventDisableTiming);
  if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&e->cap, cudaStreamNonBlocking);
  for (int q = 0; q < n && err == cudaSuccess; ++q) {
    cudaStream_t L = nullptr;
    cudaEvent_t v = nullptr;
    err = cudaStreamCreateWithFlags(&L, cudaStreamNonBlocking);
    if (err == cudaSuccess) e->lane.push_back(L);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&v, cudaEventDisableTiming);
    if (err == cudaSuccess) e->ev.push_back(v);
    for (int b = 0; b < 2 && err == cudaSuccess; ++b)
      for (int f = 0; f < 5 && err == cudaSuccess; ++f) {
        void *p = nullptr;
        err = cudaMalloc(&p, field_count(members[q]->D, f) * e->es);
        if (err == cudaSuccess) e->buf[b].push_back(p);
      }
  }
  if (err != cudaSuccess) {
    e->release();
    delete e;
    return cuda_fail(err, "ensemble buffers");
  }
  *out = e;
  return EB_OK;
}

eb_status eb_ensemble_destroy(eb_ensemble e) {
  if (!e) return EB_OK;
  cudaDeviceSynchronize();
  e->release();
  delete e;
  return EB_OK;
}

eb_status eb_ensemble_set_state(eb_ensemble e, int member, const eb_state *U, void *stream) {
  if (!member_ok(e, member)) return fail(EB_ERR_INVALID_ARG, "NULL ensemble or member out of range");
  if (!state_ok(U, e->es)) return fail(EB_ERR_INVALID_ARG, "state pointer NULL or misaligned");
  cudaStream_t s = as_stream(stream);
  eb_geom g = e->m[member];
  void **u = state_ptrs(U);
  void *cur[5], *other[5];
  for (int f = 0; f < 5; ++f) {
    cur[f] = e->field(e->cur, member, f);
    other[f] = e->field(1 - e->cur, member, f);
    CUDA_TRY(cudaMemcpyAsync(cur[f], u[f], field_count(g->D, f) * e->es, cudaMemcpyDeviceToDevice, s), "load state");
  }
  // covered CVs and the w wall levels never change: give the other buffer
  // their values once, so the captured steps skip the pass-through
  if (e->prec == EB_F64) launch_static_copy(step_args<double>(g, cur, cur, other, 0.0, 1), s);
  else launch_static_copy(step_args<float>(g, cur, cur, other, 0.0, 1), s);
  CUDA_TRY(cudaGetLastError(), "load state");
  return EB_OK;
}

eb_status eb_ensemble_get_state(eb_ensemble e, int member, eb_state *U, void *stream) {
  if (!member_ok(e, member)) return fail(EB_ERR_INVALID_ARG, "NULL ensemble or member out of range");
  if (!state_ok(U, e->es)) return fail(EB_ERR_INVALID_ARG, "state pointer NULL or misaligned");
  cudaStream_t s = as_stream(stream);
  void **u = state_ptrs(U);
  for (int f = 0; f < 5; ++f)
    CUDA_TRY(cudaMemcpyAsync(u[f], e->field(e->cur, member, f), field_count(e->m[member]->D, f) * e->es,
                             cudaMemcpyDeviceToDevice, s),
             "store state");
  return EB_OK;
}

eb_status eb_ensemble_step(eb_ensemble e, const double *dt, int nsteps, void *stream) {
  if (!e) return fail(EB_ERR_INVALID_ARG, "NULL ensemble");
  if (!dt) return fail(EB_ERR_INVALID_ARG, "dt is NULL");
  if (nsteps < 0) return fail(EB_ERR_INVALID_ARG, "nsteps must be >= 0");
  for (size_t q = 0; q < e->m.size(); ++q)
    if (!(dt[q] > 0.0) || !isfinite(dt[q])) return fail(EB_ERR_INVALID_ARG, "every dt must be finite and > 0");
  bool same = true;
  for (size_t q = 0; q < e->m.size(); ++q) same = same && dt[q] == e->dt[q];
  if (!same) {   // the time steps are part of the captured kernels' arguments
    e->drop_graphs();
    e->dt.assign(dt, dt + e->m.size());
  }
  return run_steps(e, nsteps, as_stream(stream));
}

eb_status eb_ensemble_tune(eb_ensemble e, const double *dt, int reps, int *slab_levels, void *stream) {
  if (!e) return fail(EB_ERR_INVALID_ARG, "NULL ensemble");
  if (!dt) return fail(EB_ERR_INVALID_ARG, "dt is NULL");
  if (reps < 1) return fail(EB_ERR_INVALID_ARG, "reps must be >= 1");
  cudaStream_t s = as_stream(stream);
  // the timed steps run on the loaded states: keep a copy and put it back
  std::vector<void *> keep;
  cudaError_t ke = cudaSuccess;
  for (size_t q = 0; q < e->m.size() && ke == cudaSuccess; ++q)
    for (int f = 0; f < 5 && ke == cudaSuccess; ++f) {
      void *p = nullptr;
      const size_t bytes = field_count(e->m[q]->D, f) * e->es;
      ke = cudaMalloc(&p, bytes);
      if (ke == cudaSuccess) {
        keep.push_back(p);
        ke = cudaMemcpyAsync(p, e->field(e->cur, (int)q, f), bytes, cudaMemcpyDeviceToDevice, s);
      }
    }
  const int cur0 = e->cur;
  auto restore = [&]() {
    e->cur = cur0;
    for (size_t q = 0, t = 0; q < e->m.size(); ++q)
      for (int f = 0; f < 5 && t < keep.size(); ++f, ++t)
        cudaMemcpyAsync(e->field(cur0, (int)q, f), keep[t], field_count(e->m[q]->D, f) * e->es,
                        cudaMemcpyDeviceToDevice, s);
    cudaStreamSynchronize(s);
    for (void *p : keep) cudaFree(p);
    for (eb_geom g : e->m) cudaMemset(g->status, 0, sizeof(unsigned));   // flags of the trial steps
  };
  if (ke != cudaSuccess) {
    restore();
    return cuda_fail(ke, "tuning snapshot");
  }
  int nzmax = 0;
  for (eb_geom g : e->m) nzmax = std::max(nzmax, g->D.nz);
  std::vector<int> cand = {0, 8, 16, 24, 32, 48, 64};
  if (nzmax > 64) cand.push_back(nzmax);
  cudaEvent_t t0, t1;
  CUDA_TRY(cudaEventCreate(&t0), "event");
  CUDA_TRY(cudaEventCreate(&t1), "event");
  float best = 0.f;
  int best_c = 0, best_h = 0;
  bool first = true;
  eb_status st = EB_OK;
  for (int c : cand) {
    for (eb_geom g : e->m)
      if ((st = eb_replan_bulk(g, c)) != EB_OK) break;
    if (st != EB_OK) break;
    // every member's bulk kernel at the same, then at a higher stream priority
    for (int hp = 0; hp < 2 && st == EB_OK; ++hp) {
      for (eb_geom g : e->m) g->bulk_high = hp;
      e->drop_graphs();
      e->dt.assign(dt, dt + e->m.size());
      if ((st = run_steps(e, 2, s)) != EB_OK) break;   // capture both graphs, warm up
      cudaEventRecord(t0, s);
      if ((st = run_steps(e, 2 * reps, s)) != EB_OK) break;
      cudaEventRecord(t1, s);
      const cudaError_t ce = cudaEventSynchronize(t1);
      if (ce != cudaSuccess) {
        st = cuda_fail(ce, "tuning step");
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, t0, t1);
      if (first || ms < best) {
        best = ms;
        best_c = c;
        best_h = hp;
        first = false;
      }
    }
    if (st != EB_OK) break;
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  restore();
  if (st != EB_OK) return st;
  for (eb_geom g : e->m) {
    if ((st = eb_replan_bulk(g, best_c)) != EB_OK) return st;
    g->bulk_high = best_h;
  }
  e->drop_graphs();
  if (slab_levels) *slab_levels = best_c;
  return EB_OK;
}

}  // extern "C"
