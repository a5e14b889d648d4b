// eb_api.cu -- the C ABI of include/eb.h: argument checks, the geometry
// handle, and the orchestration of the kernels on the caller's stream.
#include "eb_handle.cuh"

#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#define EB_VERSION_NUM 100

namespace {
thread_local std::string g_last_error;
}  // namespace

std::string &eb_error_slot() { return g_last_error; }

eb_status eb_replan_bulk(eb_geom g, int slab_levels) {
  std::vector<int> seg, off;
  CUDA_TRY(bulk_plan(g->D, g->kfast_host.data(), g->prec == EB_F64, slab_levels, g->tile_rows, seg, off),
           "bulk work split");
  // the split arrays are small: the old ones are released right away
  for (void *p : {(void *)g->bseg, (void *)g->boff}) {
    if (!p) continue;
    for (size_t q = 0; q < g->allocs.size(); ++q)
      if (g->allocs[q] == p) {
        g->allocs.erase(g->allocs.begin() + q);
        break;
      }
    cudaFree(p);
  }
  g->bseg = nullptr;
  g->boff = nullptr;
  g->slab_levels = slab_levels;
  g->bctas = (int)off.size() - 1;
  ++g->plan_gen;
  CUDA_TRY(g->alloc(&g->bseg, std::max<long long>(1, (long long)seg.size() / 4)), "alloc bulk split");
  CUDA_TRY(g->alloc(&g->boff, (long long)off.size()), "alloc bulk split");
  if (!seg.empty())
    CUDA_TRY(cudaMemcpy(g->bseg, seg.data(), sizeof(int) * seg.size(), cudaMemcpyHostToDevice), "copy bulk split");
  CUDA_TRY(cudaMemcpy(g->boff, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice), "copy bulk split");
  return EB_OK;
}

using namespace ebh;

namespace {

bool bad_desc(const eb_desc *d, std::string &why) {
  if (!d) { why = "desc is NULL"; return true; }
  if (d->nx < 4 || d->ny < 4 || d->nz < 4) { why = "nx, ny, nz must be >= 4"; return true; }
  if ((long long)d->nx * d->ny * (d->nz + 1) >= (1LL << 32)) {
    why = "grid too large: nx*ny*(nz+1) must be below 2^32";
    return true;
  }
  if (!(d->Lx > 0) || !(d->Ly > 0) || !(d->Lz > 0) || !isfinite(d->Lx) || !isfinite(d->Ly) || !isfinite(d->Lz)) {
    why = "Lx, Ly, Lz must be finite and > 0";
    return true;
  }
  if (!(d->v_target_frac > 0.0) || !(d->v_target_frac <= 1.0)) { why = "v_target_frac must lie in (0, 1]"; return true; }
  return false;
}

// A per-level profile is stored with PROFILE_PAD zero levels on both sides
// (the pointer kept is that of level 0), so the bulk kernel reads levels
// -PROFILE_PAD .. nz + PROFILE_PAD - 1 without bounds checks.
constexpr int PROFILE_PAD = 4;

template <typename P>
cudaError_t alloc_profile(eb_geom g, P **p) {
  const int n = g->D.nz + 2 * PROFILE_PAD;
  P *base = nullptr;
  cudaError_t e = g->alloc(&base, n);
  if (e != cudaSuccess) return e;
  e = cudaMemset(base, 0, sizeof(P) * n);
  *p = base + PROFILE_PAD;
  return e;
}

template <typename T>
cudaError_t fill_ref(eb_geom g, const double *src, double **dd, float **ff, cudaStream_t s) {
  const int nz = g->D.nz;
  std::vector<double> hv(nz, 0.0);
  if (src) {
    cudaError_t e = cudaMemcpyAsync(hv.data(), src, sizeof(double) * nz, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
  }
  std::vector<float> hf(nz);
  for (int k = 0; k < nz; ++k) hf[k] = (float)hv[k];
  cudaError_t e = alloc_profile(g, dd);
  if (e != cudaSuccess) return e;
  e = alloc_profile(g, ff);
  if (e != cudaSuccess) return e;
  e = cudaMemcpy(*dd, hv.data(), sizeof(double) * nz, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*ff, hf.data(), sizeof(float) * nz, cudaMemcpyHostToDevice);
}

// Background advected values of every level from the reference profiles
// (device copies in g->ref_d): theta0 = ref_rt / ref_rho, u_bg = ref_u /
// ref_rho, v_bg = ref_v / ref_rho, in double, with their float copies; zero
// on levels whose reference density is zero (no profile given).
cudaError_t update_background(eb_geom g) {
  const int nz = g->D.nz;
  std::vector<double> r[4];
  for (int q = 0; q < 4; ++q) {
    r[q].resize(nz);
    cudaError_t e = cudaMemcpy(r[q].data(), g->ref_d[q], sizeof(double) * nz, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return e;
  }
  for (int b = 0; b < 3; ++b) {
    std::vector<double> hd(nz);
    std::vector<float> hf(nz);
    for (int k = 0; k < nz; ++k) {
      hd[k] = r[0][k] > 0.0 ? r[b + 1][k] / r[0][k] : 0.0;
      hf[k] = (float)hd[k];
    }
    cudaError_t e = cudaMemcpy(g->bg_d[b], hd.data(), sizeof(double) * nz, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->bg_f[b], hf.data(), sizeof(float) * nz, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Builds the handle's geometry, tables and lists: from the nodal heights, or
// (fine != nullptr) as the coarse level of the fine handle, merged from its
// cells (eb_amr.cu; the heights then are every other fine node, kept as a
// record of the terrain).
eb_status build_impl(eb_geom g, const double *h_nodes, const double *ref_rho, const double *ref_rt, cudaStream_t s,
                     eb_geom fine = nullptr) {
  g->has_ref = ref_rho != nullptr;
  const Dims &D = g->D;
  const long long ncol = (long long)D.nx * D.ny;
  const long long nh = (long long)(D.nx + 1) * (D.ny + 1);
  CUDA_TRY(g->alloc(&g->h, nh), "alloc heights");
  if (fine) launch_subsample_heights(fine->h, fine->D, g->h, D, s);
  else CUDA_TRY(cudaMemcpyAsync(g->h, h_nodes, sizeof(double) * nh, cudaMemcpyDeviceToDevice, s), "copy heights");
  long long *counts = nullptr;
  long long scan_room = 2 * (ncol + 2) + 8;
  CUDA_TRY(g->alloc(&counts, scan_room), "alloc counts");
  long long nrec[4];
  for (int q = 0; q < 4; ++q) {
    CUDA_TRY(g->alloc(&g->kcov[q], ncol), "alloc kcov");
    CUDA_TRY(g->alloc(&g->kreg[q], ncol), "alloc kreg");
    CUDA_TRY(g->alloc(&g->kxt[q], ncol), "alloc kxt");
    CUDA_TRY(g->alloc(&g->roff[q], ncol + 1), "alloc roff");
    if (fine) launch_coarse_bounds(fine->D, fine->G[0], D, q, g->kcov[q], g->kreg[q], s);
    else launch_band_bounds(g->h, D, q, g->kcov[q], g->kreg[q], s);
  }
  for (int q = 0; q < 4; ++q) {
    const int nzg = nzg_of(D, q);
    CUDA_TRY(cudaMemsetAsync(g->roff[q], 0, sizeof(long long) * (ncol + 1), s), "memset roff");
    launch_band_top(D, nzg, g->kcov[q], g->kreg[q], g->kxt[q], g->roff[q], s);
    scan_exclusive(g->roff[q], ncol + 1, counts, s);
    CUDA_TRY(cudaMemcpyAsync(&nrec[q], counts, sizeof(long long), cudaMemcpyDeviceToHost, s), "read nrec");
  }
  CUDA_TRY(cudaGetLastError(), "band kernels");
  CUDA_TRY(cudaStreamSynchronize(s), "band sync");
  long long tmp_need = 0;
  for (int q = 0; q < 4; ++q) {
    GridDev &G = g->G[q];
    G.nzg = nzg_of(D, q);
    G.kcov = g->kcov[q];
    G.kxt = g->kxt[q];
    G.roff = g->roff[q];
    G.nrec = nrec[q];
    const long long n = nrec[q];
    g->info.band_records[q] = n;
    CUDA_TRY(g->alloc(&G.alpha, n), "alloc geometry");
    CUDA_TRY(g->alloc(&G.cent, 3 * n), "alloc geometry");
    CUDA_TRY(g->alloc(&G.beta, 3 * n), "alloc geometry");
    CUDA_TRY(g->alloc(&G.fcent, 6 * n), "alloc geometry");
    CUDA_TRY(g->alloc(&G.nrm, 3 * n), "alloc geometry");
    CUDA_TRY(g->alloc(&G.aeb, n), "alloc geometry");
    CUDA_TRY(g->alloc(&G.ebc, 3 * n), "alloc geometry");
    CUDA_TRY(g->alloc(&G.flag, n), "alloc geometry");
    CUDA_TRY(g->alloc(&G.alpha_f, n), "alloc geometry");
    CUDA_TRY(g->alloc(&G.beta_f, 3 * n), "alloc geometry");
    CUDA_TRY(g->alloc(&G.fcent_f, 6 * n), "alloc geometry");
    CUDA_TRY(g->alloc(&G.code, n), "alloc tables");
    CUDA_TRY(g->alloc(&G.nnb, n), "alloc tables");
    CUDA_TRY(g->alloc(&G.kappa, n), "alloc tables");
    CUDA_TRY(g->alloc(&G.omega, n), "alloc tables");
    CUDA_TRY(g->alloc(&G.vhat, n), "alloc tables");
    CUDA_TRY(g->alloc(&G.xhat, 3 * n), "alloc tables");
    if (fine) launch_coarse_geometry(fine->D, fine->G[0], D, q, G, s);
    else launch_band_geometry(g->h, D, q, G, s);
    tmp_need = std::max(tmp_need, 2 * (n + 1) + 1 + (n + 1) / 256 + 8);
  }
  CUDA_TRY(cudaGetLastError(), "geometry kernels");
  // first level of the bulk kernel per column, from the regular and fluid
  // levels of all grids
  {
    CUDA_TRY(g->alloc(&g->kfast, ncol), "alloc kfast");
    int *kflu = nullptr;
    CUDA_TRY(cudaMalloc(&kflu, sizeof(int) * (size_t)(4 * ncol)), "alloc fluid levels");
    const int *kr[4] = {g->kreg[0], g->kreg[1], g->kreg[2], g->kreg[3]};
    const int *kfl[4] = {kflu, kflu + ncol, kflu + 2 * ncol, kflu + 3 * ncol};
    for (int q = 0; q < 4; ++q) launch_fluid_level(D, g->G[q], kflu + q * ncol, s);
    launch_fast_level(D, kr, kfl, g->kfast, s);
    const cudaError_t e = cudaStreamSynchronize(s);
    cudaFree(kflu);
    CUDA_TRY(e, "fast levels");
  }
  // dense availability bytes and the near-EB update lists
  std::vector<int> kf_host(ncol);
  CUDA_TRY(cudaMemcpy(kf_host.data(), g->kfast, sizeof(int) * ncol, cudaMemcpyDeviceToHost), "read kfast");
  int kmax = 0;
  for (long long c = 0; c < ncol; ++c) kmax = std::max(kmax, kf_host[c]);
  if ((long long)D.nxy * (D.nz + 1) >= (1LL << 32)) return fail(EB_ERR_INVALID_ARG, "grid too large for 32-bit lists");
  {
    long long *mark = nullptr;
    const long long nm = std::max(1LL, D.nxy * (long long)kmax);
    CUDA_TRY(cudaMalloc(&mark, sizeof(long long) * (size_t)(nm + 1)), "alloc band marks");
    long long *scan_tmp = nullptr;
    cudaError_t e = cudaMalloc(&scan_tmp, sizeof(long long) * (size_t)(nm / 256 + 16));
    if (e != cudaSuccess) { cudaFree(mark); return cuda_fail(e, "alloc band scan"); }
    for (int q = 0; q < 4 && e == cudaSuccess; ++q) {
      GridDev &G = g->G[q];
      e = g->alloc(&G.dflag, D.nxy * nzg_of(D, q));
      if (e != cudaSuccess) break;
      launch_dense_flags(D, q, G, s);
      long long nb = 0;
      if (kmax > 0) {
        e = cudaMemsetAsync(mark, 0, sizeof(long long) * (size_t)(nm + 1), s);
        launch_band_marks(D, q, g->kcov[q], g->kfast, kmax, mark, s);
        scan_exclusive(mark, nm + 1, scan_tmp, s);
        e = cudaMemcpyAsync(&nb, scan_tmp, sizeof(long long), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
      }
      G.nband = nb;
      if (e == cudaSuccess) e = g->alloc(&G.blist, nb);
      if (e == cudaSuccess && nb > 0) launch_band_fill(D, q, g->kcov[q], g->kfast, kmax, mark, G.blist, s);
    }
    cudaStreamSynchronize(s);
    cudaFree(mark);
    cudaFree(scan_tmp);
    if (e != cudaSuccess) return cuda_fail(e, "band lists");
  }
  // each band list: the cut CVs, which take a row of coefficients, first;
  // then the regular ones, with or without a record (all faces open, centroids
  // at the face centres: plain face differences, a shorter kernel); plane
  // order kept
  {
    std::vector<int> kx(ncol), kc(ncol);
    std::vector<long long> ro(ncol + 1);
    std::vector<uint8_t> fl;
    std::vector<unsigned> bl, ord;
    for (int q = 0; q < 4; ++q) {
      GridDev &G = g->G[q];
      G.nband_rec = 0;
      if (G.nband == 0) continue;
      bl.resize(G.nband);
      fl.resize(std::max(1LL, G.nrec));
      CUDA_TRY(cudaMemcpy(bl.data(), G.blist, sizeof(unsigned) * G.nband, cudaMemcpyDeviceToHost), "read band list");
      CUDA_TRY(cudaMemcpy(kx.data(), g->kxt[q], sizeof(int) * ncol, cudaMemcpyDeviceToHost), "read kxt");
      CUDA_TRY(cudaMemcpy(kc.data(), g->kcov[q], sizeof(int) * ncol, cudaMemcpyDeviceToHost), "read kcov");
      CUDA_TRY(cudaMemcpy(ro.data(), g->roff[q], sizeof(long long) * (ncol + 1), cudaMemcpyDeviceToHost), "read roff");
      if (G.nrec)
        CUDA_TRY(cudaMemcpy(fl.data(), G.flag, sizeof(uint8_t) * G.nrec, cudaMemcpyDeviceToHost), "read flags");
      auto takes_row = [&](unsigned c) {
        const long long k = c / D.nxy, col = c % D.nxy;
        return k < kx[col] && fl[ro[col] + (k - kc[col])] != EBK_REGULAR;
      };
      ord.clear();
      for (int pass = 0; pass < 2; ++pass)
        for (unsigned c : bl)
          if (takes_row(c) == (pass == 0)) ord.push_back(c);
      for (unsigned c : bl)
        if (takes_row(c)) ++G.nband_rec;
      CUDA_TRY(cudaMemcpy(G.blist, ord.data(), sizeof(unsigned) * G.nband, cudaMemcpyHostToDevice), "write band list");
    }
  }
  // faces whose provisional fluxes the near-EB path reads (they lie below
  // kfast + 2), and the dense arrays those fluxes are staged in
  {
    const int kface = std::min(D.nz + 1, kmax + 2);
    const long long nfa = std::max(1LL, D.nxy * (long long)kface);
    const size_t es = g->prec == EB_F64 ? sizeof(double) : sizeof(float);
    uint8_t *mk[3] = {nullptr, nullptr, nullptr};
    long long *cnt = nullptr, *scan_tmp = nullptr;
    cudaError_t e = cudaSuccess;
    for (int d = 0; d < 3 && e == cudaSuccess; ++d) e = cudaMalloc(&mk[d], (size_t)nfa);
    if (e == cudaSuccess) e = cudaMalloc(&cnt, sizeof(long long) * (size_t)(nfa + 1));
    if (e == cudaSuccess) e = cudaMalloc(&scan_tmp, sizeof(long long) * (size_t)(nfa / 256 + 16));
    for (int q = 0; q < 4 && e == cudaSuccess; ++q) {
      GridDev &G = g->G[q];
      for (int d = 0; d < 3; ++d) e = e == cudaSuccess ? cudaMemsetAsync(mk[d], 0, (size_t)nfa, s) : e;
      if (e != cudaSuccess) break;
      launch_face_marks(D, q, G, mk[0], mk[1], mk[2], s);
      for (int d = 0; d < 3 && e == cudaSuccess; ++d) {
        e = cudaMemsetAsync(cnt, 0, sizeof(long long) * (size_t)(nfa + 1), s);
        launch_marks_to_counts(mk[d], nfa, cnt, s);
        scan_exclusive(cnt, nfa + 1, scan_tmp, s);
        long long nf = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&nf, scan_tmp, sizeof(long long), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        G.nface[d] = nf;
        if (e == cudaSuccess) e = g->alloc(&G.flist[d], nf);
        if (e == cudaSuccess && nf > 0) launch_marks_fill(mk[d], nfa, cnt, G.flist[d], s);
        if (e == cudaSuccess) e = g->alloc(&G.fmask[d], nf);
        if (e == cudaSuccess) e = g->alloc((char **)&G.fh[d], (long long)(nfa * es));
        G.fhm[d] = nullptr;
        if (e == cudaSuccess && q == 0) e = g->alloc((char **)&G.fhm[d], (long long)(nfa * es));
      }
    }
    if (e == cudaSuccess) {
      launch_face_masks(D, g->G, s);
      e = cudaStreamSynchronize(s);
    }
    // FP64 path: the CVs whose advected values the face stencils read, staged
    // once per step (the float path forms them per face)
    uint8_t *sm[4] = {nullptr, nullptr, nullptr, nullptr};
    long long nsm[4] = {0, 0, 0, 0};
    const bool staging = g->prec == EB_F64;
    for (int q = 0; q < 4; ++q) {
      g->G[q].nstage = 0;
      g->G[q].stlist = nullptr;
      g->G[q].pv = nullptr;
    }
    for (int q = 0; q < 4 && e == cudaSuccess && staging; ++q) {
      g->G[q].nst = std::min(nzg_of(D, q), kface + 1);
      nsm[q] = std::max(1LL, D.nxy * (long long)g->G[q].nst);
      e = cudaMalloc(&sm[q], (size_t)nsm[q]);
      if (e == cudaSuccess) e = cudaMemsetAsync(sm[q], 0, (size_t)nsm[q], s);
    }
    long long *cnt2 = nullptr, *tmp2 = nullptr;
    long long nmax = std::max(std::max(nsm[0], nsm[1]), std::max(nsm[2], nsm[3]));
    if (e == cudaSuccess) e = cudaMalloc(&cnt2, sizeof(long long) * (size_t)(nmax + 1));
    if (e == cudaSuccess) e = cudaMalloc(&tmp2, sizeof(long long) * (size_t)(nmax / 256 + 16));
    if (e == cudaSuccess && staging) launch_stage_marks(D, g->G, sm, s);
    for (int q = 0; q < 4 && e == cudaSuccess && staging; ++q) {
      GridDev &G = g->G[q];
      e = cudaMemsetAsync(cnt2, 0, sizeof(long long) * (size_t)(nsm[q] + 1), s);
      launch_marks_to_counts(sm[q], nsm[q], cnt2, s);
      scan_exclusive(cnt2, nsm[q] + 1, tmp2, s);
      long long n = 0;
      if (e == cudaSuccess) e = cudaMemcpyAsync(&n, tmp2, sizeof(long long), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      G.nstage = n;
      if (e == cudaSuccess) e = g->alloc(&G.stlist, n);
      if (e == cudaSuccess && n > 0) launch_marks_fill(sm[q], nsm[q], cnt2, G.stlist, s);
      if (e == cudaSuccess) e = g->alloc((char **)&G.pv, (long long)(nsm[q] * es));
      if (e == cudaSuccess) e = cudaMemsetAsync(G.pv, 0, (size_t)nsm[q] * es, s);   // never-staged CVs read 0
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (int q = 0; q < 4; ++q) cudaFree(sm[q]);
    cudaFree(cnt2);
    cudaFree(tmp2);
    for (int d = 0; d < 3; ++d) cudaFree(mk[d]);
    cudaFree(cnt);
    cudaFree(scan_tmp);
    if (e != cudaSuccess) return cuda_fail(e, "face lists");
  }
  // near-EB rows of the CVs with a record: count, scan, allocate, fill
  for (int q = 0; q < 4; ++q) {
    GridDev &G = g->G[q];
    const long long nr = G.nband_rec;
    const long long n = 3 * nr + 1;
    long long *cnt = nullptr, *scan_tmp = nullptr;
    cudaError_t e = cudaMalloc(&cnt, sizeof(long long) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&scan_tmp, sizeof(long long) * (size_t)(n / 256 + 16));
    long long nt = 0;
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(long long) * (size_t)n, s);
    if (e == cudaSuccess) {
      launch_band_rows(D, g->G, q, false, cnt, s);
      scan_exclusive(cnt, n, scan_tmp, s);
      e = cudaMemcpyAsync(&nt, scan_tmp, sizeof(long long), cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && nt >= (1LL << 32)) {
      cudaFree(cnt);
      cudaFree(scan_tmp);
      return fail(EB_ERR_INVALID_ARG, "near-EB rows exceed 2^32 terms");
    }
    G.nterm = nt;
    if (e == cudaSuccess) e = g->alloc(&G.srow, n);
    if (e == cudaSuccess) e = g->alloc(&G.sidx, nt);
    if (e == cudaSuccess) e = g->alloc(&G.scoef, nt);
    if (e == cudaSuccess) e = g->alloc(&G.scoef_f, nt);
    if (e == cudaSuccess) e = g->alloc(&G.stiny, nr);
    if (e == cudaSuccess) {
      launch_band_rows(D, g->G, q, true, cnt, s);
      launch_rows_to_u32(cnt, n, G.srow, s);
      e = cudaStreamSynchronize(s);
    }
    cudaFree(cnt);
    cudaFree(scan_tmp);
    if (e != cudaSuccess) return cuda_fail(e, "near-EB rows");
  }
  long long *tmp = nullptr;
  CUDA_TRY(g->alloc(&tmp, tmp_need), "alloc set-up scratch");
  for (int q = 0; q < 4; ++q) {
    cudaError_t e = build_wsrd(D, q, g->G[q], g->G, g->desc.v_target_frac, g->W[q], s, tmp);
    if (e != cudaSuccess) return cuda_fail(e, "redistribution set-up");
    g->max_small = std::max(g->max_small, g->W[q].nsmall);
    g->info.small_cvs[q] = g->W[q].nsmall;
    g->info.affected_cvs[q] = g->W[q].naff;
  }
  // the redistribution may run beside the bulk kernel when every CV it reads
  // or writes is produced by the near-EB kernels
  {
    unsigned *far = nullptr, far_h = 1;
    CUDA_TRY(cudaMalloc(&far, sizeof(unsigned)), "alloc reach flag");
    cudaError_t e = cudaMemsetAsync(far, 0, sizeof(unsigned), s);
    for (int q = 0; q < 4 && e == cudaSuccess; ++q) launch_wsrd_reach(D, q, g->W[q], g->kcov[q], g->kfast, far, s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&far_h, far, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(far);
    CUDA_TRY(e, "redistribution reach");
    g->wsrd_side = far_h == 0 ? 1 : 0;
  }
  CUDA_TRY(g->alloc((double **)&g->qhat, g->max_small), "alloc qhat");
  CUDA_TRY(g->alloc((double **)&g->sig, 3 * g->max_small), "alloc sig");
  CUDA_TRY(g->alloc((double **)&g->pval, g->max_small), "alloc pivot values");
  g->sum_small = 2 * g->W[0].nsmall + g->W[1].nsmall + g->W[2].nsmall + g->W[3].nsmall;
  CUDA_TRY(g->alloc((double **)&g->qhat5, g->sum_small), "alloc qhat");
  CUDA_TRY(g->alloc((double **)&g->sig5, 3 * g->sum_small), "alloc sig");
  CUDA_TRY(g->alloc((double **)&g->pval5, g->sum_small), "alloc pivot values");
  {
    int least = 0, greatest = 0;
    CUDA_TRY(cudaDeviceGetStreamPriorityRange(&least, &greatest), "stream priorities");
    CUDA_TRY(cudaStreamCreateWithPriority(&g->bulk, cudaStreamNonBlocking, greatest), "bulk stream");
    CUDA_TRY(cudaStreamCreateWithFlags(&g->side, cudaStreamNonBlocking), "side stream");
  }
  CUDA_TRY(cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming), "event");
  CUDA_TRY(cudaEventCreateWithFlags(&g->ev_join, cudaEventDisableTiming), "event");
  CUDA_TRY(cudaEventCreateWithFlags(&g->ev_join_bulk, cudaEventDisableTiming), "event");
  CUDA_TRY(fill_ref<double>(g, ref_rho, &g->ref_d[0], &g->ref_f[0], s), "reference");
  CUDA_TRY(fill_ref<double>(g, ref_rt, &g->ref_d[1], &g->ref_f[1], s), "reference");
  CUDA_TRY(fill_ref<double>(g, nullptr, &g->ref_d[2], &g->ref_f[2], s), "reference");
  CUDA_TRY(fill_ref<double>(g, nullptr, &g->ref_d[3], &g->ref_f[3], s), "reference");
  for (int q = 0; q < 3; ++q) {
    CUDA_TRY(alloc_profile(g, &g->bg_d[q]), "alloc background");
    CUDA_TRY(alloc_profile(g, &g->bg_f[q]), "alloc background");
  }
  CUDA_TRY(update_background(g), "background");
  CUDA_TRY(g->alloc(&g->status, 1), "alloc status");
  CUDA_TRY(cudaMemsetAsync(g->status, 0, sizeof(unsigned), s), "memset status");
  // host-side counts for eb_geom_info
  std::vector<int> kc(ncol), kf(ncol);
  CUDA_TRY(cudaMemcpy(kf.data(), g->kfast, sizeof(int) * ncol, cudaMemcpyDeviceToHost), "read kfast");
  g->kfast_host = kf;
  {
    const eb_status st = eb_replan_bulk(g, 0);
    if (st != EB_OK) return st;
  }
  g->info.cells = (int64_t)ncol * D.nz;
  g->info.fast_cells = 0;
  for (long long c = 0; c < ncol; ++c) g->info.fast_cells += D.nz - std::min(kf[c], D.nz);
  double amin = 1.0;
  for (int q = 0; q < 4; ++q) {
    CUDA_TRY(cudaMemcpy(kc.data(), g->kcov[q], sizeof(int) * ncol, cudaMemcpyDeviceToHost), "read kcov");
    const int nzg = nzg_of(D, q);
    int64_t cvs = 0, band = 0;
    for (long long c = 0; c < ncol; ++c) {
      cvs += nzg - kc[c];
      for (int k = kc[c]; k < std::min(kf[c], nzg); ++k)
        if (!(q == 3 && (k == 0 || k == D.nz))) ++band;
    }
    g->info.cvs[q] = cvs;
    g->info.band_cvs[q] = band;
    g->info.band_faces[q] = g->G[q].nface[0] + g->G[q].nface[1] + g->G[q].nface[2];
    for (long long c = 0; c < ncol; ++c) g->kcov_max = std::max(g->kcov_max, kc[c]);
    {
      // pass-through list: covered CVs level by level, then (w grid) the walls
      std::vector<unsigned> st;
      const int k0 = q == 3 ? 1 : 0, k1 = q == 3 ? D.nz : nzg;
      for (int k = k0; k < k1; ++k)
        for (long long c = 0; c < ncol; ++c)
          if (k < kc[c]) st.push_back((unsigned)(c + D.nxy * k));
      if (q == 3)
        for (int k : {0, D.nz})
          for (long long c = 0; c < ncol; ++c) st.push_back((unsigned)(c + D.nxy * k));
      GridDev &G = g->G[q];
      G.nstatic = (long long)st.size();
      CUDA_TRY(g->alloc(&G.slist, G.nstatic), "alloc pass-through list");
      if (G.nstatic)
        CUDA_TRY(cudaMemcpy(G.slist, st.data(), sizeof(unsigned) * st.size(), cudaMemcpyHostToDevice),
                 "write pass-through list");
    }
    const long long n = nrec[q];
    std::vector<double> al(n > 0 ? n : 1);
    std::vector<uint8_t> fl(n > 0 ? n : 1);
    if (n > 0) {
      CUDA_TRY(cudaMemcpy(al.data(), g->G[q].alpha, sizeof(double) * n, cudaMemcpyDeviceToHost), "read alpha");
      CUDA_TRY(cudaMemcpy(fl.data(), g->G[q].flag, n, cudaMemcpyDeviceToHost), "read flag");
    }
    int64_t tiny = 0;
    for (long long r = 0; r < n; ++r) {
      if (fl[r] == EBK_CUT && al[r] > 0.0 && al[r] < 1e-3) ++tiny;
      if (al[r] > 0.0 && al[r] < amin) amin = al[r];
    }
    g->info.tiny_cvs[q] = tiny;
  }
  g->info.min_alpha = amin;
  return EB_OK;
}


}  // namespace

// Scratch of eb_wsrd_noalloc.  It is part of the library's device image, so
// using it allocates nothing; there is one block per device, shared by every
// handle, which is why overlapping calls race.
static __device__ __align__(256) unsigned char g_wsrd_noalloc_scratch[EB_WSRD_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kNoallocMaxDevices] = {};
unsigned long long g_noalloc_ctx[kNoallocMaxDevices] = {};

// Unique id of the calling thread's current CUDA context (never reused within
// the process, unlike a context handle), through the driver entry points that
// the runtime hands out, so the library needs no link to libcuda.  0 when the
// driver does not provide it.
unsigned long long current_context_id() {
  using GetCurrent = int (*)(void **);
  using GetId = int (*)(void *, unsigned long long *);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *a = nullptr, *b = nullptr;
    cudaDriverEntryPointQueryResult qa, qb;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) == cudaSuccess &&
        qa == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) == cudaSuccess &&
        qb == cudaDriverEntryPointSuccess) {
      get_current = reinterpret_cast<GetCurrent>(a);
      get_id = reinterpret_cast<GetId>(b);
    }
  });
  void *ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
  return id;
}

// Device address of the fixed scratch on `device`, which must be current.
// Looked up once per device and context: a context torn down and created
// again (cudaDeviceReset by the application or another library) loads the
// library's device image afresh, so its address is looked up again.
eb_status noalloc_scratch(int device, void **out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (device < 0 || device >= kNoallocMaxDevices) return fail(EB_ERR_INVALID_ARG, "device index out of range");
  const unsigned long long ctx = current_context_id();
  if (!g_noalloc_addr[device] || ctx == 0 || ctx != g_noalloc_ctx[device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_wsrd_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "address of the fixed redistribution scratch");
    g_noalloc_addr[device] = p;
    g_noalloc_ctx[device] = ctx;
  }
  *out = g_noalloc_addr[device];
  return EB_OK;
}

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

// Same launches as wsrd_field, with the three per-small-CV arrays carved out
// of `scratch`: deviation sums, pivot values, then 3 slopes per small CV.
template <typename T>
void wsrd_field_scratch(eb_geom g, int field, T *u, char *scratch, cudaStream_t s) {
  const int grid = field <= 1 ? 0 : field - 1;
  const size_t one = round256((size_t)g->W[grid].nsmall * sizeof(T));
  WsrdArgs<T> R;
  R.D = g->D;
  R.W = g->W[grid];
  R.u = u;
  R.refd = field <= 3 ? g->ref_d[field] : nullptr;
  R.dev = (T *)scratch;
  R.pval = (T *)(scratch + one);
  R.sig = (T *)(scratch + 2 * one);
  R.status = g->status;
  launch_wsrd(R, s);
}

}  // namespace

extern "C" {

static eb_status build_common(const eb_desc *desc, const double *h_nodes, eb_precision prec, const double *ref_rho,
                              const double *ref_rhotheta, void *stream, eb_geom *out, eb_geom fine) {
  eb_geom g = new eb_geom_s();
  memset(&g->info, 0, sizeof(g->info));
  g->desc = *desc;
  g->prec = prec;
  cudaGetDevice(&g->device);
  g->D.nx = desc->nx;
  g->D.ny = desc->ny;
  g->D.nz = desc->nz;
  g->D.nxy = (long long)desc->nx * desc->ny;
  g->D.dx = desc->Lx / desc->nx;
  g->D.dy = desc->Ly / desc->ny;
  g->D.dz = desc->Lz / desc->nz;
  g->D.fnx.init((unsigned)desc->nx);
  g->D.fny.init((unsigned)desc->ny);
  g->D.fnxy.init((unsigned)g->D.nxy);
  for (const FastDiv *f : {&g->D.fnx, &g->D.fny, &g->D.fnxy}) {   // spot check of the multipliers
    const unsigned probe[6] = {0u, f->d - 1, f->d, 2 * f->d + 1, 0x7fffffffu, 0xffffffffu};
    for (unsigned n : probe)
      if (f->div(n) != n / f->d) {
        delete g;
        return fail(EB_ERR_INVALID_ARG, "internal: fixed-divisor multiplier check failed");
      }
  }
  g->D.idx = 1.0 / g->D.dx;
  g->D.idy = 1.0 / g->D.dy;
  g->D.idz = 1.0 / g->D.dz;
  eb_status st = build_impl(g, h_nodes, ref_rho, ref_rhotheta, as_stream(stream), fine);
  if (st != EB_OK) {
    cudaStreamSynchronize(as_stream(stream));
    g->release();
    delete g;
    return st;
  }
  *out = g;
  g_last_error.clear();
  return EB_OK;
}

eb_status eb_geom_build(const eb_desc *desc, const double *h_nodes, eb_precision prec, const double *ref_rho,
                        const double *ref_rhotheta, void *stream, eb_geom *out) {
  std::string why;
  if (!out) return fail(EB_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (bad_desc(desc, why)) return fail(EB_ERR_INVALID_ARG, "%s", why.c_str());
  if (!h_nodes || ((uintptr_t)h_nodes % 8)) return fail(EB_ERR_INVALID_ARG, "h_nodes is NULL or misaligned");
  if (prec != EB_F64 && prec != EB_MIXED) return fail(EB_ERR_INVALID_ARG, "unknown precision");
  if ((ref_rho == nullptr) != (ref_rhotheta == nullptr))
    return fail(EB_ERR_INVALID_ARG, "ref_rho and ref_rhotheta must both be given or both be NULL");
  return build_common(desc, h_nodes, prec, ref_rho, ref_rhotheta, stream, out, nullptr);
}

eb_status eb_geom_build_coarse(eb_geom fine, const double *ref_rho, const double *ref_rhotheta, void *stream,
                               eb_geom *out) {
  std::string why;
  if (!out) return fail(EB_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!fine) return fail(EB_ERR_INVALID_ARG, "NULL fine handle");
  if (fine->D.nx % 2 || fine->D.ny % 2 || fine->D.nz % 2)
    return fail(EB_ERR_INVALID_ARG, "the fine level needs even nx, ny and nz");
  eb_desc desc = fine->desc;
  desc.nx /= 2;
  desc.ny /= 2;
  desc.nz /= 2;
  if (bad_desc(&desc, why)) return fail(EB_ERR_INVALID_ARG, "%s", why.c_str());
  if ((ref_rho == nullptr) != (ref_rhotheta == nullptr))
    return fail(EB_ERR_INVALID_ARG, "ref_rho and ref_rhotheta must both be given or both be NULL");
  int cur = -1;
  CUDA_TRY(cudaGetDevice(&cur), "current device");
  if (cur != fine->device) return fail(EB_ERR_INVALID_ARG, "the current device is not the fine handle's device");
  return build_common(&desc, nullptr, fine->prec, ref_rho, ref_rhotheta, stream, out, fine);
}

eb_status eb_geom_destroy(eb_geom geom) {
  if (!geom) return EB_OK;
  cudaDeviceSynchronize();
  geom->release();
  delete geom;
  return EB_OK;
}

eb_status eb_geom_info(eb_geom geom, eb_geom_info_t *info) {
  if (!geom || !info) return fail(EB_ERR_INVALID_ARG, "NULL handle or info");
  *info = geom->info;
  info->slab_levels = geom->slab_levels;
  info->bulk_high_priority = geom->bulk_high;
  info->wsrd_beside_bulk = geom->wsrd_side;
  info->tile_rows = geom->tile_rows;
  return EB_OK;
}

eb_status eb_geom_export(eb_geom geom, eb_grid grid, eb_export_field field, double *dst, void *stream) {
  if (!geom) return fail(EB_ERR_INVALID_ARG, "NULL handle");
  if ((int)grid < 0 || (int)grid > 3) return fail(EB_ERR_INVALID_ARG, "unknown grid");
  if ((int)field < 0 || (int)field >= EB_X_COUNT) return fail(EB_ERR_INVALID_ARG, "unknown export field");
  if (!dst || ((uintptr_t)dst % 8)) return fail(EB_ERR_INVALID_ARG, "dst is NULL or misaligned");
  launch_export_geometry(geom->h, geom->D, (int)grid, geom->G[grid], (int)field, dst, as_stream(stream));
  CUDA_TRY(cudaGetLastError(), "export");
  return EB_OK;
}

eb_status eb_flux_div(eb_geom geom, const eb_state *U, eb_state *dU, void *stream) {
  if (!geom) return fail(EB_ERR_INVALID_ARG, "NULL handle");
  const size_t al = geom->prec == EB_F64 ? 8 : 4;
  if (!state_ok(U, al) || !state_ok(dU, al)) return fail(EB_ERR_INVALID_ARG, "state pointer NULL or misaligned");
  void **u = state_ptrs(U), **d = state_ptrs(dU);
  for (int f = 0; f < 5; ++f)
    for (int e = 0; e < 5; ++e)
      if (u[f] == d[e]) return fail(EB_ERR_INVALID_ARG, "U and dU overlap");
  if (geom->prec == EB_F64) flux_update(geom, step_args<double>(geom, u, nullptr, d, 1.0, 1), as_stream(stream));
  else flux_update(geom, step_args<float>(geom, u, nullptr, d, 1.0, 1), as_stream(stream));
  CUDA_TRY(cudaGetLastError(), "flux divergence");
  return EB_OK;
}

eb_status eb_wsrd(eb_geom geom, eb_field field, const void *Uhat, void *Unew, void *stream) {
  if (!geom) return fail(EB_ERR_INVALID_ARG, "NULL handle");
  if ((int)field < 0 || (int)field > 4) return fail(EB_ERR_INVALID_ARG, "unknown field");
  const size_t es = geom->prec == EB_F64 ? 8 : 4;
  if (!Uhat || !Unew || ((uintptr_t)Uhat % es) || ((uintptr_t)Unew % es))
    return fail(EB_ERR_INVALID_ARG, "field pointer NULL or misaligned");
  const size_t bytes = field_count(geom->D, (int)field) * es;
  cudaStream_t s = as_stream(stream);
  if (Uhat != Unew) {
    const char *a = (const char *)Uhat, *b = (const char *)Unew;
    if (a < b + bytes && b < a + bytes) return fail(EB_ERR_INVALID_ARG, "Uhat and Unew overlap");
    CUDA_TRY(cudaMemcpyAsync(Unew, Uhat, bytes, cudaMemcpyDeviceToDevice, s), "copy field");
  }
  if (geom->prec == EB_F64) wsrd_field<double>(geom, (int)field, (double *)Unew, s);
  else wsrd_field<float>(geom, (int)field, (float *)Unew, s);
  CUDA_TRY(cudaGetLastError(), "redistribution");
  return EB_OK;
}

eb_status eb_wsrd_noalloc(eb_geom geom, eb_field field, const void *Uhat, void *Unew, void *stream) {
  if (!geom) return fail(EB_ERR_INVALID_ARG, "NULL handle");
  if ((int)field < 0 || (int)field > 4) return fail(EB_ERR_INVALID_ARG, "unknown field");
  const size_t es = geom->prec == EB_F64 ? 8 : 4;
  if (!Uhat || !Unew || ((uintptr_t)Uhat % es) || ((uintptr_t)Unew % es))
    return fail(EB_ERR_INVALID_ARG, "field pointer NULL or misaligned");
  const size_t bytes = field_count(geom->D, (int)field) * es;
  if (Uhat != Unew) {
    const char *a = (const char *)Uhat, *b = (const char *)Unew;
    if (a < b + bytes && b < a + bytes) return fail(EB_ERR_INVALID_ARG, "Uhat and Unew overlap");
  }
  int cur = -1;
  CUDA_TRY(cudaGetDevice(&cur), "current device");
  if (cur != geom->device) return fail(EB_ERR_INVALID_ARG, "the current device is not the handle's device");
  const int grid = (int)field <= 1 ? 0 : (int)field - 1;
  const size_t one = round256((size_t)geom->W[grid].nsmall * es);
  const size_t need = 2 * one + round256(3 * (size_t)geom->W[grid].nsmall * es);
  if (need > (size_t)EB_WSRD_NOALLOC_SCRATCH_BYTES) {
    char buf[256];
    snprintf(buf, sizeof(buf), "field needs %zu bytes of scratch (%lld small CVs), the fixed block holds %zu",
             need, (long long)geom->W[grid].nsmall, (size_t)EB_WSRD_NOALLOC_SCRATCH_BYTES);
    return fail(EB_ERR_INVALID_ARG, "%s", buf);
  }
  void *scratch = nullptr;
  eb_status st = noalloc_scratch(cur, &scratch);
  if (st != EB_OK) return st;
  cudaStream_t s = as_stream(stream);
  if (Uhat != Unew) CUDA_TRY(cudaMemcpyAsync(Unew, Uhat, bytes, cudaMemcpyDeviceToDevice, s), "copy field");
  if (geom->prec == EB_F64) wsrd_field_scratch<double>(geom, (int)field, (double *)Unew, (char *)scratch, s);
  else wsrd_field_scratch<float>(geom, (int)field, (float *)Unew, (char *)scratch, s);
  CUDA_TRY(cudaGetLastError(), "redistribution");
  return EB_OK;
}

eb_status eb_step(eb_geom geom, const eb_state *Un, eb_state *Unp1, double dt, int nsteps, int stages, void *stream) {
  if (!geom) return fail(EB_ERR_INVALID_ARG, "NULL handle");
  const size_t es = geom->prec == EB_F64 ? 8 : 4;
  if (!state_ok(Un, es) || !state_ok(Unp1, es)) return fail(EB_ERR_INVALID_ARG, "state pointer NULL or misaligned");
  if (!(dt > 0.0) || !isfinite(dt)) return fail(EB_ERR_INVALID_ARG, "dt must be finite and > 0");
  if (nsteps < 0) return fail(EB_ERR_INVALID_ARG, "nsteps must be >= 0");
  if (stages != 1 && stages != 3) return fail(EB_ERR_INVALID_ARG, "stages must be 1 or 3");
  void **u0 = state_ptrs(Un), **u1 = state_ptrs(Unp1);
  for (int f = 0; f < 5; ++f) {
    const size_t bytes = field_count(geom->D, f) * es;
    for (int e = 0; e < 5; ++e) {
      const size_t b2 = field_count(geom->D, e) * es;
      const char *a = (const char *)u0[f], *b = (const char *)u1[e];
      if (a < b + b2 && b < a + bytes) return fail(EB_ERR_INVALID_ARG, "Un and Unp1 overlap");
    }
  }
  cudaStream_t s = as_stream(stream);
  if (nsteps == 0) {
    for (int f = 0; f < 5; ++f)
      CUDA_TRY(cudaMemcpyAsync(u1[f], u0[f], field_count(geom->D, f) * es, cudaMemcpyDeviceToDevice, s), "copy");
    return EB_OK;
  }
  // scratch states: C, D ping-pong between steps, A, B hold Runge-Kutta stages
  const int need = stages == 3 ? 4 : 2;
  for (int b = 0; b < need; ++b)
    for (int f = 0; f < 5; ++f)
      if (!geom->scr[b][f]) {
        cudaError_t e = cudaMalloc(&geom->scr[b][f], field_count(geom->D, f) * es);
        if (e != cudaSuccess) return cuda_fail(e, "alloc step scratch");
        geom->allocs.push_back(geom->scr[b][f]);
        geom->info.device_bytes += (int64_t)(field_count(geom->D, f) * es);
      }
  void **C = geom->scr[0], **Dd = geom->scr[1], **A = geom->scr[2], **B = geom->scr[3];
  bool fresh[5] = {true, true, true, true, true};   // C, D, A, B, Unp1 need their static CVs once
  auto fresh_of = [&](void **p) -> bool & {
    return p == C ? fresh[0] : p == Dd ? fresh[1] : p == A ? fresh[2] : p == B ? fresh[3] : fresh[4];
  };
  void **cur = u0;
  for (int n = 0; n < nsteps; ++n) {
    void **dst = (n == nsteps - 1) ? u1 : (cur == C ? Dd : C);
    if (stages == 1) {
      bool &fr = fresh_of(dst);
      if (geom->prec == EB_F64) stage<double>(geom, cur, cur, dst, dt, fr, s);
      else stage<float>(geom, cur, cur, dst, dt, fr, s);
      fr = false;
    } else {
      const double c[3] = {dt / 3.0, dt / 2.0, dt};
      void **srcs[3] = {cur, A, B};
      void **outs[3] = {A, B, dst};
      for (int q = 0; q < 3; ++q) {
        bool &fr = fresh_of(outs[q]);
        if (geom->prec == EB_F64) stage<double>(geom, srcs[q], cur, outs[q], c[q], fr, s);
        else stage<float>(geom, srcs[q], cur, outs[q], c[q], fr, s);
        fr = false;
      }
    }
    cur = dst;
  }
  CUDA_TRY(cudaGetLastError(), "step");
  return EB_OK;
}

eb_status eb_step_profile(eb_geom geom, const eb_state *Un, eb_state *Unp1, double dt, void *stream, float ms[4]) {
  if (!geom || !ms) return fail(EB_ERR_INVALID_ARG, "NULL handle or ms");
  const size_t es = geom->prec == EB_F64 ? 8 : 4;
  if (!state_ok(Un, es) || !state_ok(Unp1, es)) return fail(EB_ERR_INVALID_ARG, "state pointer NULL or misaligned");
  if (!(dt > 0.0) || !isfinite(dt)) return fail(EB_ERR_INVALID_ARG, "dt must be finite and > 0");
  void **u0 = state_ptrs(Un), **u1 = state_ptrs(Unp1);
  for (int f = 0; f < 5; ++f)
    for (int e = 0; e < 5; ++e)
      if (u0[f] == u1[e]) return fail(EB_ERR_INVALID_ARG, "Un and Unp1 overlap");
  cudaStream_t s = as_stream(stream);
  cudaEvent_t ev[4];
  for (int q = 0; q < 4; ++q) CUDA_TRY(cudaEventCreate(&ev[q]), "event");
  if (geom->prec == EB_F64) {
    StepArgs<double> A = step_args<double>(geom, u0, u0, u1, dt, 1);
    launch_static_copy(A, s);
    cudaEventRecord(ev[0], s);
    launch_flux_bulk(A, s);
    cudaEventRecord(ev[1], s);
    launch_flux_band(A, s);
    cudaEventRecord(ev[2], s);
    wsrd_all<double>(geom, u1, s);
  } else {
    StepArgs<float> A = step_args<float>(geom, u0, u0, u1, dt, 1);
    launch_static_copy(A, s);
    cudaEventRecord(ev[0], s);
    launch_flux_bulk(A, s);
    cudaEventRecord(ev[1], s);
    launch_flux_band(A, s);
    cudaEventRecord(ev[2], s);
    wsrd_all<float>(geom, u1, s);
  }
  cudaEventRecord(ev[3], s);
  cudaError_t e = cudaEventSynchronize(ev[3]);
  if (e == cudaSuccess) {
    cudaEventElapsedTime(&ms[0], ev[0], ev[1]);
    cudaEventElapsedTime(&ms[1], ev[1], ev[2]);
    cudaEventElapsedTime(&ms[2], ev[2], ev[3]);
    cudaEventElapsedTime(&ms[3], ev[0], ev[3]);
  }
  for (int q = 0; q < 4; ++q) cudaEventDestroy(ev[q]);
  CUDA_TRY(e, "profiled step");
  return EB_OK;
}

eb_status eb_geom_set_tile_rows(eb_geom geom, int rows) {
  if (!geom) return fail(EB_ERR_INVALID_ARG, "NULL handle");
  if (rows != 16 && rows != 14) return fail(EB_ERR_INVALID_ARG, "rows must be 16 or 14");
  if (rows == 14 && geom->prec == EB_F64) return fail(EB_ERR_INVALID_ARG, "14-row tiles are for the mixed path");
  CUDA_TRY(cudaDeviceSynchronize(), "drain before re-planning");
  geom->tile_rows = rows;
  return eb_replan_bulk(geom, geom->slab_levels);
}

eb_status eb_geom_set_slab_levels(eb_geom geom, int slab_levels) {
  if (!geom) return fail(EB_ERR_INVALID_ARG, "NULL handle");
  if (slab_levels < 0) return fail(EB_ERR_INVALID_ARG, "slab_levels must be >= 0");
  CUDA_TRY(cudaDeviceSynchronize(), "drain before re-planning");
  return eb_replan_bulk(geom, slab_levels);
}

eb_status eb_geom_set_wind_reference(eb_geom geom, const double *ref_rhou, const double *ref_rhov, void *stream) {
  if (!geom) return fail(EB_ERR_INVALID_ARG, "NULL handle");
  if (!geom->has_ref && (ref_rhou || ref_rhov))
    return fail(EB_ERR_STATE, "a momentum profile needs a handle built with a reference density profile");
  const int nz = geom->D.nz;
  cudaStream_t s = as_stream(stream);
  std::vector<double> hv[2];
  const double *src[2] = {ref_rhou, ref_rhov};
  bool nonzero = false;
  for (int q = 0; q < 2; ++q) {
    hv[q].assign(nz, 0.0);
    if (src[q]) {
      if ((uintptr_t)src[q] % 8) return fail(EB_ERR_INVALID_ARG, "reference profile pointer misaligned");
      CUDA_TRY(cudaMemcpyAsync(hv[q].data(), src[q], sizeof(double) * nz, cudaMemcpyDeviceToHost, s),
               "read momentum profile");
    }
  }
  CUDA_TRY(cudaStreamSynchronize(s), "read momentum profile");
  for (int q = 0; q < 2; ++q)
    for (int k = 0; k < nz; ++k) {
      if (!isfinite(hv[q][k])) return fail(EB_ERR_INVALID_ARG, "momentum profile holds a non-finite value");
      nonzero = nonzero || hv[q][k] != 0.0;
    }
  // the handle's work on its own streams reads the profiles: let it finish
  CUDA_TRY(cudaDeviceSynchronize(), "drain before replacing the momentum profile");
  for (int q = 0; q < 2; ++q) {
    std::vector<float> hf(nz);
    for (int k = 0; k < nz; ++k) hf[k] = (float)hv[q][k];
    CUDA_TRY(cudaMemcpy(geom->ref_d[2 + q], hv[q].data(), sizeof(double) * nz, cudaMemcpyHostToDevice),
             "write momentum profile");
    CUDA_TRY(cudaMemcpy(geom->ref_f[2 + q], hf.data(), sizeof(float) * nz, cudaMemcpyHostToDevice),
             "write momentum profile");
  }
  geom->has_wind_ref = nonzero;
  CUDA_TRY(update_background(geom), "background");
  return EB_OK;
}

eb_status eb_geom_set_sources(eb_geom geom, int flags) {
  if (!geom) return fail(EB_ERR_INVALID_ARG, "NULL handle");
  if (flags & ~(EB_SOURCE_PRESSURE | EB_SOURCE_BUOYANCY)) return fail(EB_ERR_INVALID_ARG, "unknown source flags");
  if (flags && !geom->has_ref)
    return fail(EB_ERR_STATE, "the sources need a handle built with the reference profiles rho0 and rho0*theta0");
  if (flags && !geom->src_d[0]) {
    // per-level tables from the reference: p0 (equation of state of rho0
    // theta0) and 1 / (rho0 theta0), in double and in float
    const int nz = geom->D.nz;
    std::vector<double> rt(nz), td[2];
    CUDA_TRY(cudaMemcpy(rt.data(), geom->ref_d[1], sizeof(double) * nz, cudaMemcpyDeviceToHost), "read profile");
    const double gamma = EB_CP / (EB_CP - EB_RD);
    for (int q = 0; q < 2; ++q) td[q].resize(nz);
    for (int k = 0; k < nz; ++k) {
      if (!(rt[k] > 0.0)) return fail(EB_ERR_STATE, "the reference rho0*theta0 must be positive for the sources");
      td[0][k] = EB_P00 * pow(EB_RD * rt[k] / EB_P00, gamma);
      td[1][k] = 1.0 / rt[k];
    }
    for (int q = 0; q < 2; ++q) {
      std::vector<float> tf(td[q].begin(), td[q].end());
      CUDA_TRY(geom->alloc(&geom->src_d[q], nz), "alloc source tables");
      CUDA_TRY(geom->alloc(&geom->src_f[q], nz), "alloc source tables");
      CUDA_TRY(cudaMemcpy(geom->src_d[q], td[q].data(), sizeof(double) * nz, cudaMemcpyHostToDevice), "tables");
      CUDA_TRY(cudaMemcpy(geom->src_f[q], tf.data(), sizeof(float) * nz, cudaMemcpyHostToDevice), "tables");
    }
  }
  if (flags && !geom->src_pp) {
    const size_t es = geom->prec == EB_F64 ? sizeof(double) : sizeof(float);
    double *pp = nullptr;   // one cell field in the state's precision
    CUDA_TRY(geom->alloc(&pp, (long long)((geom->D.nxy * geom->D.nz * es + 7) / 8)), "alloc source scratch");
    geom->src_pp = pp;
  }
  geom->src_flags = flags;
  return EB_OK;
}

eb_status eb_geom_set_bulk_priority(eb_geom geom, int high) {
  if (!geom) return fail(EB_ERR_INVALID_ARG, "NULL handle");
  if (high != 0 && high != 1) return fail(EB_ERR_INVALID_ARG, "high must be 0 or 1");
  geom->bulk_high = high;
  return EB_OK;
}

eb_status eb_geom_tune(eb_geom geom, const eb_state *U, double dt, int reps, int *slab_levels, void *stream) {
  if (!geom) return fail(EB_ERR_INVALID_ARG, "NULL handle");
  const size_t es = geom->prec == EB_F64 ? 8 : 4;
  if (!state_ok(U, es)) return fail(EB_ERR_INVALID_ARG, "state pointer NULL or misaligned");
  if (!(dt > 0.0) || !isfinite(dt)) return fail(EB_ERR_INVALID_ARG, "dt must be finite and > 0");
  if (reps < 1) return fail(EB_ERR_INVALID_ARG, "reps must be >= 1");
  cudaStream_t s = as_stream(stream);
  // the trial steps write into a handle-owned state (allocated here)
  void *out[5] = {};
  for (int f = 0; f < 5; ++f) {
    const cudaError_t e = cudaMalloc(&out[f], field_count(geom->D, f) * es);
    if (e != cudaSuccess) {
      for (int q = 0; q < f; ++q) cudaFree(out[q]);
      return cuda_fail(e, "alloc tuning state");
    }
  }
  eb_state O;
  void **op = state_ptrs(&O);
  for (int f = 0; f < 5; ++f) op[f] = out[f];
  std::vector<int> cand = {0, 12, 16, 24, 32, 48, 64};
  if (geom->D.nz > 64) cand.push_back(geom->D.nz);
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  float best = 0.f;
  int best_c = 0, best_h = 0, best_r = 16;
  bool first = true;
  eb_status st = EB_OK;
  const int rows_cand[2] = {16, 14};
  const int nrows = geom->prec == EB_F64 ? 1 : 2;
  for (int ri = 0; ri < nrows && st == EB_OK; ++ri)
  for (int c : cand) {
    geom->tile_rows = rows_cand[ri];
    if ((st = eb_replan_bulk(geom, c)) != EB_OK) break;
    for (int hp = 0; hp < 2 && st == EB_OK; ++hp) {
      geom->bulk_high = hp;
      if ((st = eb_step(geom, U, &O, dt, 1, 1, stream)) != EB_OK) break;   // warm-up
      cudaEventRecord(t0, s);
      for (int q = 0; q < reps && st == EB_OK; ++q) st = eb_step(geom, U, &O, dt, 1, 1, stream);
      cudaEventRecord(t1, s);
      if (st != EB_OK) break;
      const cudaError_t e = cudaEventSynchronize(t1);
      if (e != cudaSuccess) {
        st = cuda_fail(e, "tuning step");
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, t0, t1);
      if (first || ms < best) {
        best = ms;
        best_c = c;
        best_h = hp;
        best_r = rows_cand[ri];
        first = false;
      }
    }
    if (st != EB_OK) break;
  }
  geom->bulk_high = best_h;
  geom->tile_rows = best_r;
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  cudaStreamSynchronize(s);
  for (int f = 0; f < 5; ++f) cudaFree(out[f]);
  cudaMemset(geom->status, 0, sizeof(unsigned));   // flags of the trial steps
  if (st != EB_OK) return st;
  if ((st = eb_replan_bulk(geom, best_c)) != EB_OK) return st;
  if (slab_levels) *slab_levels = best_c;
  return EB_OK;
}

eb_status eb_sync_status(eb_geom geom, void *stream) {
  if (!geom) return fail(EB_ERR_INVALID_ARG, "NULL handle");
  cudaStream_t s = as_stream(stream);
  CUDA_TRY(cudaStreamSynchronize(s), "synchronise");
  unsigned w = 0;
  CUDA_TRY(cudaMemcpy(&w, geom->status, sizeof(unsigned), cudaMemcpyDeviceToHost), "read status");
  CUDA_TRY(cudaMemset(geom->status, 0, sizeof(unsigned)), "clear status");
  if (w & EB_DEV_TIMEOUT) return fail(EB_ERR_TIMEOUT, "a bounded device-side wait expired");
  if (w & EB_DEV_NUMERIC) return fail(EB_ERR_NUMERIC, "a kernel produced a non-finite value");
  return EB_OK;
}

const char *eb_last_error(void) { return g_last_error.c_str(); }

int eb_version(void) { return EB_VERSION_NUM; }

}  // extern "C"
