// eb_kernels.cuh -- host-side launch wrappers shared between the library's
// translation units.  Not part of the ABI.
#pragma once

#include "eb_internal.cuh"

#include <vector>

// Compact redistribution tables of one grid (Sec. 5.1), built once.
struct WsrdDev {
  long long nsmall = 0, naff = 0, nlsq = 0, nw = 0;
  int *sid = nullptr;             // [nrec] small id of a record, -1 if not small
  // per small CV
  long long *s_lin = nullptr;     // state index
  long long *s_rec = nullptr;     // record
  int *s_nmem = nullptr;          // members incl. itself (<= 8)
  int *s_piv = nullptr;           // pivot member of the deviation form
  long long *s_plin = nullptr;    // state index of the pivot member
  long long *s_mlin = nullptr;    // [8 * nsmall] member state indices (slot 0: itself)
  double *s_mw = nullptr;         // [8 * nsmall] Qhat weights (sum 1)
  double *s_me = nullptr;         // [24 * nsmall] member centroid - xhat (limiter points)
  long long *s_loff = nullptr;    // [nsmall + 1] LSQ stencil offsets
  long long *l_lin = nullptr;     // [nlsq] stencil CV state index
  int *l_sid = nullptr;           // [nlsq] small id of the stencil CV or -1
  long long *l_plin = nullptr;    // [nlsq] pivot state index of that small CV, else the CV's own index
  double *l_c = nullptr;          // [3 * nlsq] gradient coefficient rows
  // per affected CV
  long long *a_lin = nullptr;
  int *a_sid = nullptr;           // own small id or -1
  double *a_eself = nullptr;      // [3 * naff] own centroid - own xhat
  long long *a_woff = nullptr;    // [naff + 1]
  int *w_sid = nullptr;           // [nw] small CV r whose neighbourhood holds the CV
  double *w_k = nullptr;          // [nw] kappa_r / N_i
  double *w_e = nullptr;          // [3 * nw] x_i - xhat_r (cell units, relative to r)
  // float copies of the weight tables for the mixed-precision path
  float *s_mw_f = nullptr, *s_me_f = nullptr, *l_c_f = nullptr, *a_eself_f = nullptr, *w_k_f = nullptr,
        *w_e_f = nullptr;
};

// eb_geom.cu
void launch_band_bounds(const double *h, const Dims &D, int g, int *kcov, int *kreg, cudaStream_t s);
void launch_band_top(const Dims &D, int nzg, const int *kcov, const int *kreg, int *kxt, long long *count,
                     cudaStream_t s);
void launch_fluid_level(const Dims &D, const GridDev &G, int *kflu, cudaStream_t s);
void launch_fast_level(const Dims &D, const int *const kreg[4], const int *const kflu[4], int *kfast,
                       cudaStream_t s);
void launch_band_geometry(const double *h, const Dims &D, int g, const GridDev &G, cudaStream_t s);
// two-level refinement (eb_amr.cu): band bounds and geometry records of a
// coarse level (Dc) merged from the c grid of the fine level (Df, Gf), and
// its nodal heights as every other fine node
void launch_coarse_bounds(const Dims &Df, const GridDev &Gf, const Dims &Dc, int g, int *kcov, int *kreg,
                          cudaStream_t s);
void launch_coarse_geometry(const Dims &Df, const GridDev &Gf, const Dims &Dc, int g, const GridDev &Gc,
                            cudaStream_t s);
void launch_subsample_heights(const double *hf, const Dims &Df, double *hc, const Dims &Dc, cudaStream_t s);
void launch_dense_flags(const Dims &D, int g, const GridDev &G, cudaStream_t s);
void launch_band_marks(const Dims &D, int g, const int *kcov, const int *kfast, int kmax, long long *mark,
                       cudaStream_t s);
void launch_band_fill(const Dims &D, int g, const int *kcov, const int *kfast, int kmax, const long long *pos,
                      unsigned *list, cudaStream_t s);
void launch_face_marks(const Dims &D, int g, const GridDev &G, uint8_t *m0, uint8_t *m1, uint8_t *m2, cudaStream_t s);
void launch_marks_to_counts(const uint8_t *m, long long n, long long *cnt, cudaStream_t s);
void launch_marks_fill(const uint8_t *m, long long n, const long long *pos, unsigned *list, cudaStream_t s);
void launch_export_geometry(const double *h, const Dims &D, int g, const GridDev &G, int field, double *dst,
                            cudaStream_t s);

// eb_step.cu: near-EB rows of grid g (CVs with a record), two passes: the
// term count of every (row, direction) segment into cnt[3t + d], then (after
// the scan of cnt and the allocation of G[g].sidx / scoef / scoef_f / stiny)
// the terms themselves at the scanned offsets
void launch_band_rows(const Dims &D, const GridDev G[4], int g, bool fill, long long *cnt, cudaStream_t s);
void launch_rows_to_u32(const long long *src, long long n, unsigned *dst, cudaStream_t s);
// eb_step.cu: availability bits of every listed face into G[q].fmask[d]
void launch_face_masks(const Dims &D, const GridDev G[4], cudaStream_t s);
// eb_step.cu: marks[q][idx] = 1 for every CV of grid q a listed face's
// stencil reads (marks[q] covers levels below G[q].nst)
void launch_stage_marks(const Dims &D, const GridDev G[4], uint8_t *const marks[4], cudaStream_t s);

// eb_fast.cu: split of the bulk kernel's (tile, level) work into lockstep
// slabs of slab_levels levels (0: chosen from the GPU's size); seg holds
// (tile, first level, end level, 0) per piece, off[b] .. off[b+1] the pieces
// of CTA b
cudaError_t bulk_plan(const Dims &D, const int *kfast_host, bool f64, int slab_levels, int tile_rows,
                      std::vector<int> &seg, std::vector<int> &off);

// eb_scan.cu: in-place exclusive scan of n values; total written to *total (device)
void scan_exclusive(long long *data, long long n, long long *total, cudaStream_t s);

// eb_wsrd_setup.cu
struct SetupScratch;
cudaError_t build_wsrd(const Dims &D, int g, GridDev &G, const GridDev *all, double vt, WsrdDev &W,
                       cudaStream_t s, long long *dev_tmp);
void free_wsrd(WsrdDev &W);
// sets *far when a CV the redistribution of grid g reads or writes is not a
// near-EB CV (see k_wsrd_reach)
void launch_wsrd_reach(const Dims &D, int g, const WsrdDev &W, const int *kcov, const int *kfast, unsigned *far,
                       cudaStream_t s);

// device allocation helper that tracks every pointer for one release
struct DevArena;
