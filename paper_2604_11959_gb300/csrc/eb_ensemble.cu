// eb_ensemble.cu -- many independent EB instances advanced together.
//
// An ensemble holds geometry handles of any sizes (one precision, one
// device) and two state buffers per member.  One forward-Euler step of every
// member runs in one of two schedules, both captured once per step
// direction as a CUDA graph that eb_ensemble_step replays (the two buffers
// alternating), both giving every member exactly what eb_step gives it:
//   persistent: ONE cooperative launch of k_ensemble_step (eb_step.cu),
//     whose CTAs (as many as fit the device at once) take the bulk kernel's
//     work units of all members, longest first, then the near-EB and
//     redistribution phases of all members, with bounded grid-wide barriers
//     between the phases;
//   branches: each member's own kernels (bulk, near-EB, redistribution) on
//     a branch of its own, forked from and joined to the launching stream,
//     so that the kernels of different members run side by side.
// The autotuner times whole-ensemble steps over the schedules, the slab
// height of the bulk kernel's tiles and (branches) the bulk kernel's stream
// priority, keeps the fastest and restores the states afterwards.
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
  cudaStream_t cap = nullptr;   // the graphs are captured here (the caller's stream may be the legacy one)
  size_t es = 4;
  int schedule = EB_ENSEMBLE_PERSISTENT;
  std::vector<cudaStream_t> lane;   // branches: one stream and join event per member
  std::vector<cudaEvent_t> ev;
  cudaEvent_t ev_root = nullptr;
  int ctas = 0;                 // CTAs of the persistent kernel (all resident at once)
  bool vec = true;              // every member's rows suit 16-byte copies
  // device tables of the persistent kernel, rebuilt with the graphs
  void *dmem[2] = {nullptr, nullptr};   // EnsMember<T>[n] per step direction
  int2 *units = nullptr;
  long long *pre = nullptr;             // 5 prefix arrays of n + 1 entries
  unsigned *ctl = nullptr;              // barrier and work counters
  int *fault = nullptr;                 // failure test: CTA + 1 that skips the first barrier
  int nunits = 0;
  int kinfo[3] = {0, 0, 0};             // registers per thread, static and local bytes of the kernel
  std::vector<int> gens;                // members' work-split generations the tables were built for
  EnsembleArgs<float> Ef[2];
  EnsembleArgs<double> Ed[2];

  void *field(int b, int q, int f) { return buf[b][5 * q + f]; }
  void drop_graphs() {
    for (int b = 0; b < 2; ++b)
      if (exec[b]) {
        cudaGraphExecDestroy(exec[b]);
        exec[b] = nullptr;
      }
  }
  void drop_tables() {
    for (int b = 0; b < 2; ++b) {
      if (dmem[b]) cudaFree(dmem[b]);
      dmem[b] = nullptr;
    }
    if (units) cudaFree(units);
    if (pre) cudaFree(pre);
    units = nullptr;
    pre = nullptr;
  }
  void release() {
    drop_graphs();
    drop_tables();
    if (ctl) cudaFree(ctl);
    if (fault) cudaFree(fault);
    ctl = nullptr;
    fault = nullptr;
    if (cap) cudaStreamDestroy(cap);
    for (cudaStream_t q : lane) cudaStreamDestroy(q);
    for (cudaEvent_t q : ev) cudaEventDestroy(q);
    if (ev_root) cudaEventDestroy(ev_root);
    lane.clear();
    ev.clear();
    ev_root = nullptr;
    for (int b = 0; b < 2; ++b)
      for (void *p : buf[b]) cudaFree(p);
    buf[0].clear();
    buf[1].clear();
  }
};

namespace {

// The persistent kernel's tables for the current work split and time
// steps: per step direction every member's step and redistribution
// arguments, the bulk work units of all members (one per CTA group of each
// member's own split, longest first) and the prefix sums of every phase's
// item counts.
template <typename T>
eb_status build_tables(eb_ensemble e, EnsembleArgs<T> E[2]) {
  e->drop_tables();
  const int n = (int)e->m.size();
  e->gens.resize(n);
  for (int q = 0; q < n; ++q) e->gens[q] = e->m[q]->plan_gen;
  std::vector<EnsMember<T>> host(n);
  for (int b = 0; b < 2; ++b) {
    for (int q = 0; q < n; ++q) {
      void *src[5], *dst[5];
      for (int f = 0; f < 5; ++f) {
        src[f] = e->field(b, q, f);
        dst[f] = e->field(1 - b, q, f);
      }
      host[q].A = step_args<T>(e->m[q], src, src, dst, e->dt[q], 0);
      host[q].S = wsrd_set<T>(e->m[q], dst);
    }
    CUDA_TRY(cudaMalloc(&e->dmem[b], sizeof(EnsMember<T>) * n), "ensemble tables");
    CUDA_TRY(cudaMemcpy(e->dmem[b], host.data(), sizeof(EnsMember<T>) * n, cudaMemcpyHostToDevice),
             "ensemble tables");
  }
  // bulk units: CTA group u of member q marches the pieces of its split
  struct Unit {
    int q, g;
    long long len;
  };
  std::vector<Unit> us;
  for (int q = 0; q < n; ++q) {
    eb_geom g = e->m[q];
    std::vector<int> seg, off;
    CUDA_TRY(bulk_plan(g->D, g->kfast_host.data(), g->prec == EB_F64, g->slab_levels, 16, seg, off), "work split");
    if ((int)off.size() - 1 != g->bctas)
      return fail(EB_ERR_STATE, "a member's work split changed outside the ensemble; tune it again");
    for (int u = 0; u + 1 < (int)off.size(); ++u) {
      long long len = 0;
      for (int p = off[u]; p < off[u + 1]; ++p) len += seg[4 * p + 2] - seg[4 * p + 1] + 3;
      us.push_back({q, u, len});
    }
  }
  std::stable_sort(us.begin(), us.end(), [](const Unit &a, const Unit &b) { return a.len > b.len; });
  std::vector<int2> hu(us.size());
  for (size_t u = 0; u < us.size(); ++u) hu[u] = make_int2(us[u].q, us[u].g);
  e->nunits = (int)hu.size();
  CUDA_TRY(cudaMalloc(&e->units, sizeof(int2) * std::max<size_t>(1, hu.size())), "ensemble units");
  if (!hu.empty())
    CUDA_TRY(cudaMemcpy(e->units, hu.data(), sizeof(int2) * hu.size(), cudaMemcpyHostToDevice), "ensemble units");
  // prefix sums: staged CVs, faces, near-EB CVs, small CVs and affected CVs of the five fields
  std::vector<long long> pre(5 * (n + 1), 0);
  for (int q = 0; q < n; ++q) {
    const EnsMember<T> &M = host[q];
    long long c[5] = {0, 0, 0, M.S.off_small[5], M.S.off_aff[5]};
    for (int g = 0; g < 4; ++g) {
      c[0] += M.A.G[g].nstage;
      c[2] += M.A.G[g].nband;
      for (int d = 0; d < 3; ++d) c[1] += M.A.G[g].nface[d];
    }
    for (int k = 0; k < 5; ++k) pre[k * (n + 1) + q + 1] = pre[k * (n + 1) + q] + c[k];
  }
  CUDA_TRY(cudaMalloc(&e->pre, sizeof(long long) * pre.size()), "ensemble prefixes");
  CUDA_TRY(cudaMemcpy(e->pre, pre.data(), sizeof(long long) * pre.size(), cudaMemcpyHostToDevice),
           "ensemble prefixes");
  for (int b = 0; b < 2; ++b) {
    EnsembleArgs<T> &A = E[b];
    A.m = (const EnsMember<T> *)e->dmem[b];
    A.nm = n;
    A.units = e->units;
    A.nunits = e->nunits;
    A.pre_stage = e->pre;
    A.pre_face = e->pre + (n + 1);
    A.pre_band = e->pre + 2 * (n + 1);
    A.pre_small = e->pre + 3 * (n + 1);
    A.pre_aff = e->pre + 4 * (n + 1);
    A.ctl = e->ctl;
    A.fault = e->fault;
    A.spin_limit = 1u << 20;   // about a second of polls a microsecond apart
    A.faces_first = pre[n] == 0 ? 1 : 0;   // no staged values: the face fluxes need no phase of their own
  }
  return EB_OK;
}

// Branches schedule: member q's stage (bulk, near-EB and redistribution
// kernels, the redistribution after the join of the bulk kernel).
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
// on the ensemble's stream: the counters' reset and the persistent kernel,
// or every member's stage on its own branch.
eb_status capture(eb_ensemble e, int from, cudaGraphExec_t *out) {
  cudaStream_t s = e->cap;
  cudaGraph_t graph = nullptr;
  CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "begin capture");
  cudaError_t le = cudaSuccess;
  if (e->schedule == EB_ENSEMBLE_PERSISTENT) {
    cudaMemsetAsync(e->ctl, 0, 4 * sizeof(unsigned), s);
    le = e->prec == EB_F64 ? launch_ensemble_step<double>(e->Ed[from], e->vec, e->ctas, s)
                           : launch_ensemble_step<float>(e->Ef[from], e->vec, e->ctas, s);
  } else {
    cudaEventRecord(e->ev_root, s);
    for (size_t q = 0; q < e->m.size(); ++q) {
      cudaStream_t L = e->lane[q];
      cudaStreamWaitEvent(L, e->ev_root, 0);
      if (e->prec == EB_F64) member_stage<double>(e, (int)q, from, L);
      else member_stage<float>(e, (int)q, from, L);
      cudaEventRecord(e->ev[q], L);
      cudaStreamWaitEvent(s, e->ev[q], 0);
    }
  }
  const cudaError_t ce = cudaStreamEndCapture(s, &graph);
  if (le != cudaSuccess || ce != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(le != cudaSuccess ? le : ce, "capture of the ensemble step");
  }
  const cudaError_t ie = cudaGraphInstantiate(out, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) return cuda_fail(ie, "instantiate step graph");
  return EB_OK;
}

eb_status run_steps(eb_ensemble e, int nsteps, cudaStream_t s) {
  // a member's work split rebuilt since the tables were made (eb_geom_tune,
  // eb_geom_set_slab_levels) moves its arrays: capture again
  for (size_t q = 0; q < e->gens.size(); ++q)
    if (e->gens[q] != e->m[q]->plan_gen) {
      e->drop_graphs();
      e->gens.clear();
      break;
    }
  if (nsteps > 0 && !e->exec[0] && !e->exec[1]) {
    const eb_status st = e->prec == EB_F64 ? build_tables<double>(e, e->Ed) : build_tables<float>(e, e->Ef);
    if (st != EB_OK) return st;
  }
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
  for (int q = 0; q < n; ++q) {
    if (!members[q]) return fail(EB_ERR_INVALID_ARG, "a member handle is NULL");
    if (members[q]->src_flags)
      return fail(EB_ERR_STATE, "ensembles take no compressible sources: a member has them switched on");
  }
  // the persistent kernel marches tiles of 16 rows: members keep that height
  for (int q = 0; q < n; ++q)
    if (members[q]->tile_rows != 16) {
      members[q]->tile_rows = 16;
      const eb_status st = eb_replan_bulk(members[q], members[q]->slab_levels);
      if (st != EB_OK) return st;
    }
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
  for (int q = 0; q < n; ++q) e->vec = e->vec && members[q]->D.nx % (int)(16 / e->es) == 0;
  e->ctas = e->prec == EB_F64 ? ensemble_kernel_ctas<double>(e->vec, e->kinfo)
                              : ensemble_kernel_ctas<float>(e->vec, e->kinfo);
  if (e->ctas < 1) {
    delete e;
    return fail(EB_ERR_STATE, "the device cannot hold the persistent ensemble kernel");
  }
  cudaError_t err = cudaStreamCreateWithFlags(&e->cap, cudaStreamNonBlocking);
  if (err == cudaSuccess) err = cudaEventCreateWithFlags(&e->ev_root, cudaEventDisableTiming);
  for (int q = 0; q < n && err == cudaSuccess; ++q) {
    cudaStream_t L = nullptr;
    cudaEvent_t v = nullptr;
    err = cudaStreamCreateWithFlags(&L, cudaStreamNonBlocking);
    if (err == cudaSuccess) e->lane.push_back(L);
    if (err == cudaSuccess) err = cudaEventCreateWithFlags(&v, cudaEventDisableTiming);
    if (err == cudaSuccess) e->ev.push_back(v);
  }
  if (err == cudaSuccess) err = cudaMalloc(&e->ctl, 4 * sizeof(unsigned));
  if (err == cudaSuccess) err = cudaMalloc(&e->fault, sizeof(int));
  if (err == cudaSuccess) err = cudaMemset(e->fault, 0, sizeof(int));
  for (int q = 0; q < n && err == cudaSuccess; ++q) {
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
  int best_c = 0, best_h = 0, best_s = EB_ENSEMBLE_PERSISTENT;
  bool first = true;
  eb_status st = EB_OK;
  for (int c : cand) {
    for (eb_geom g : e->m)
      if ((st = eb_replan_bulk(g, c)) != EB_OK) break;
    if (st != EB_OK) break;
    // the persistent kernel, then the branches with every member's bulk
    // kernel at the same and at a higher stream priority
    for (int v = 0; v < 3 && st == EB_OK; ++v) {
      const int sched = v == 0 ? EB_ENSEMBLE_PERSISTENT : EB_ENSEMBLE_BRANCHES;
      const int hp = v == 2 ? 1 : 0;
      e->schedule = sched;
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
        best_s = sched;
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
  e->schedule = best_s;
  e->drop_graphs();
  if (slab_levels) *slab_levels = best_c;
  return EB_OK;
}

eb_status eb_ensemble_set_schedule(eb_ensemble e, int schedule) {
  if (!e) return fail(EB_ERR_INVALID_ARG, "NULL ensemble");
  if (schedule != EB_ENSEMBLE_PERSISTENT && schedule != EB_ENSEMBLE_BRANCHES)
    return fail(EB_ERR_INVALID_ARG, "unknown schedule");
  if (schedule != e->schedule) {
    e->schedule = schedule;
    e->drop_graphs();
  }
  return EB_OK;
}

eb_status eb_ensemble_inject_barrier_fault(eb_ensemble e, int cta) {
  if (!e) return fail(EB_ERR_INVALID_ARG, "NULL ensemble");
  if (cta < -1 || cta >= e->ctas) return fail(EB_ERR_INVALID_ARG, "cta must be -1 or a CTA of the step kernel");
  const int v = cta + 1;
  CUDA_TRY(cudaDeviceSynchronize(), "drain before the fault switch");
  CUDA_TRY(cudaMemcpy(e->fault, &v, sizeof(int), cudaMemcpyHostToDevice), "fault switch");
  return EB_OK;
}

eb_status eb_ensemble_info(eb_ensemble e, int out[6]) {
  if (!e) return fail(EB_ERR_INVALID_ARG, "NULL ensemble");
  if (!out) return fail(EB_ERR_INVALID_ARG, "out is NULL");
  out[0] = e->ctas;
  out[1] = e->nunits;
  for (int q = 0; q < 3; ++q) out[2 + q] = e->kinfo[q];
  out[5] = e->schedule;
  return EB_OK;
}

}  // extern "C"
