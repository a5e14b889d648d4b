/*
 * eb_oracle.c -- plain FP64 CPU oracle for the explicit embedded-boundary (EB)
 * advance on a staggered (Arakawa C) mesh of Kang, Almgren, Natarajan et al.,
 * "An Embedded Boundary Scheme for Three-Dimensional Flow Over Terrain on a
 * Staggered Mesh".
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, import or
 * run this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header or table with the CUDA path.
 *
 * Compiled with -ffp-contract=off: no fused multiply-adds.  Every loop is a
 * plain loop over control volumes (CVs); the OpenMP pragmas only split the
 * outer loop, every CV's arithmetic is independent of the thread count.
 *
 * Contents, in the paper's order:
 *   1. geometry (Sec. 3.2): nodal level set -> cut-cell moments of the
 *      cell-centred grid, and of the three face grids as sums of two
 *      half-cells;
 *   2. fluxes and the cut-cell update (Sec. 4.1, Eqs. update-cc / update-fc,
 *      flux interpolation to the face centroid);
 *   3. weighted state redistribution (Sec. 5.1, Eqs. kappa, omega, nbhd_vol,
 *      centroid, qhat_omega, qrecon, final_update_omega);
 *   4. the sources of the compressible system (Sec. 2.1, Eq. mom-comp): the
 *      perturbation pressure gradient from the equation of state and the
 *      buoyancy, added to the flux divergence of every stage when asked for;
 *   5. the step of Algorithm 1 (stages = 1: forward Euler of Eq. FV-discrete;
 *      stages = 3: the three-stage Runge-Kutta of Sec. 5.2 with WSRD after
 *      every stage);
 *   6. two-level static refinement (Sec. 4.3): the geometry of the coarse
 *      level merged from the fine level's cells, and the restriction of a
 *      fine state (volume- and area-weighted averages).
 *
 * Units: inside the geometry every length is in grid units (x / dx, y / dy,
 * z / dz).  Volume fractions are relative to dx*dy*dz, face fractions to the
 * full face area, centroid offsets are in grid units relative to the CV (or
 * face) centre.  The unit EB normal points into the fluid, in physical space.
 *
 * Windows: every array is allocated over a window of columns
 * [x0, x0+WX) x [y0, y0+WY) of a periodic NX x NY domain, full height.  With
 * WX = NX and WY = NY the window is the whole periodic domain.  A stencil
 * access that leaves a smaller window reads as "absent"; results within a
 * margin of the window edge are then meaningless and the caller ignores them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_COVERED 0
#define ORC_REGULAR 1
#define ORC_CUT 2

enum { GC = 0, GU = 1, GV = 2, GW = 3 };

typedef struct {
  int NX, NY, nz;          /* global cells                                  */
  int x0, y0, WX, WY;      /* window of columns held by every array          */
  double dx, dy, dz;       /* cell sizes                                     */
  const double *h;         /* nodal terrain heights, (NY+1) x (NX+1), x fastest */
} OrcDomain;

/* Per-grid geometry, dense over the window; n = WX*WY*nzg. */
typedef struct {
  double *alpha;  /* n   volume fraction                                   */
  double *cent;   /* 3n  volume-centroid offset [d*n + c]                   */
  double *beta;   /* 3n  area fraction of the LOW d-face of the CV          */
  double *fcent;  /* 6n  low-face centroid offsets, transverse axes [(2d+t)*n + c] */
  double *aeb;    /* n   EB area / (dx*dy)                                  */
  double *nrm;    /* 3n  unit EB normal into the fluid (physical)           */
  double *ebc;    /* 3n  EB centroid offset                                 */
  double *ebv;    /* 3n  grid-unit EB vector sum_f a_f (-dH/dxi, -dH/deta, 1) */
  uint8_t *flag;  /* n   covered / regular / cut                            */
} OrcGeom;

/* Weighted state redistribution tables of one grid (Sec. 5.1). */
typedef struct {
  uint8_t *code;  /* n  neighbourhood code, 0 = not a small CV               */
  int *nnb;       /* n  N, number of neighbourhoods that contain the CV      */
  double *kappa;  /* n                                                        */
  double *omega;  /* n                                                        */
  double *vhat;   /* n  weighted neighbourhood volume (units of dx*dy*dz)     */
  double *xhat;   /* 3n weighted neighbourhood centroid, offset from CV centre */
} OrcWsrd;

static inline int nzg_of(const OrcDomain *D, int g) { return D->nz + (g == GW ? 1 : 0); }
static inline long ncv(const OrcDomain *D, int g) { return (long)D->WX * D->WY * nzg_of(D, g); }

static inline int imod(int a, int m) { int r = a % m; return r < 0 ? r + m : r; }

/* Window-local linear index of global (gi, gj, k) on grid g, or -1 if the
 * position is outside the window or outside the grid's vertical range. */
static long loc(const OrcDomain *D, int g, int gi, int gj, int k) {
  if (k < 0 || k >= nzg_of(D, g)) return -1;
  int li = imod(gi - D->x0, D->NX), lj = imod(gj - D->y0, D->NY);
  if (li >= D->WX || lj >= D->WY) return -1;
  return (long)li + (long)D->WX * ((long)lj + (long)D->WY * k);
}

/* ------------------------------------------------------------------------- */
/* 1. Geometry (Sec. 3.2)                                                     */
/* ------------------------------------------------------------------------- */
/*
 * The EB is the nodal level set phi = z - h at the lattice nodes, made
 * piecewise linear: each lattice square is split along its (0,0)-(1,1)
 * diagonal into T1 (xi >= eta) and T2 (eta >= xi), and h is linear on each.
 * Fluid is z > h.  Staggered CVs are unions of half-cells, so every piece of
 * geometry is a polygon whose corners lie on the half lattice {0, 1/2, 1}^2
 * of one square.  Heights there are taken as
 *   corners: h_node / dz;  edge and diagonal midpoints: (Ha + Hb) * 0.5,
 * which is also what the covered / regular classification compares against
 * the exact levels k and k + 1/2.
 */

typedef struct { double x, y, H; } Pt;

/* Heights on the 3 x 3 half lattice of square (I, J), Hq[a][b] at
 * (xi, eta) = (a/2, b/2). */
static void half_lattice(const OrcDomain *D, int I, int J, double Hq[3][3]) {
  int i0 = imod(I, D->NX), j0 = imod(J, D->NY);
  const double *h = D->h;
  long W = D->NX + 1;
  double H00 = h[(long)j0 * W + i0] / D->dz;
  double H10 = h[(long)j0 * W + i0 + 1] / D->dz;
  double H01 = h[(long)(j0 + 1) * W + i0] / D->dz;
  double H11 = h[(long)(j0 + 1) * W + i0 + 1] / D->dz;
  Hq[0][0] = H00; Hq[2][0] = H10; Hq[0][2] = H01; Hq[2][2] = H11;
  Hq[1][0] = (H00 + H10) * 0.5;
  Hq[1][2] = (H01 + H11) * 0.5;
  Hq[0][1] = (H00 + H01) * 0.5;
  Hq[2][1] = (H10 + H11) * 0.5;
  Hq[1][1] = (H00 + H11) * 0.5;
}

/* Sutherland-Hodgman clip of a convex polygon against the half plane
 * sgn*(coordinate c) <= lim (c = 0: x, 1: y).  Used only on half-lattice
 * coordinates, where every intersection is at a half-lattice point. */
static int clip_coord(const Pt *in, int n, int c, double lim, double sgn, Pt *out) {
  int m = 0;
  for (int e = 0; e < n; e++) {
    Pt p = in[e], q = in[(e + 1) % n];
    double vp = sgn * ((c == 0) ? p.x : p.y) - sgn * lim;
    double vq = sgn * ((c == 0) ? q.x : q.y) - sgn * lim;
    int pin = vp <= 0.0, qin = vq <= 0.0;
    if (pin && qin) {
      out[m++] = q;
    } else if (pin && !qin) {
      double t = vp / (vp - vq);
      Pt r = {p.x + t * (q.x - p.x), p.y + t * (q.y - p.y), 0.0};
      out[m++] = r;
    } else if (!pin && qin) {
      double t = vp / (vp - vq);
      Pt r = {p.x + t * (q.x - p.x), p.y + t * (q.y - p.y), 0.0};
      out[m++] = r;
      out[m++] = q;
    }
  }
  return m;
}

/* Clip against a level of the height: keep H < lev (below = 1) or H >= lev. */
static int clip_level(const Pt *in, int n, double lev, int below, Pt *out) {
  int m = 0;
  for (int e = 0; e < n; e++) {
    Pt p = in[e], q = in[(e + 1) % n];
    int pin = below ? (p.H < lev) : (p.H >= lev);
    int qin = below ? (q.H < lev) : (q.H >= lev);
    if (pin != qin) {
      double t = (lev - p.H) / (q.H - p.H);
      Pt r = {p.x + t * (q.x - p.x), p.y + t * (q.y - p.y), lev};
      out[m++] = r;
    }
    if (qin) out[m++] = q;
  }
  return m;
}

/* Integrals over a convex polygon of the functions needed below, by fan
 * triangulation and the three-edge-midpoint rule (exact for quadratics).
 * H is linear on each fan triangle.  The fluid height g = Z1 - H is formed
 * at the vertices and averaged to the edge midpoints, so that a thin sliver
 * of fluid (g small everywhere) keeps its relative accuracy. */
typedef struct { double a, x, y, g, xg, yg, zg; } PolyInt;
/* a = area, x = int xi, y = int eta, g = int (Z1 - H),
 * xg = int xi*g, yg = int eta*g, zg = int g*(Z1 - zb - g/2), the z-moment of
 * the fluid column [H, Z1] measured from zb */

static void poly_integrals(const Pt *p, int n, double zb, double Z1, PolyInt *s) {
  memset(s, 0, sizeof(*s));
  const double top = Z1 - zb;
  for (int t = 1; t + 1 < n; t++) {
    const Pt *v[3] = {&p[0], &p[t], &p[t + 1]};
    double A = 0.5 * ((v[1]->x - v[0]->x) * (v[2]->y - v[0]->y) -
                      (v[2]->x - v[0]->x) * (v[1]->y - v[0]->y));
    if (!(A > 0.0)) continue;
    s->a += A;
    /* g is linear: its integral is the area times the vertex mean */
    s->g += A * ((Z1 - v[0]->H) + (Z1 - v[1]->H) + (Z1 - v[2]->H)) / 3.0;
    for (int e = 0; e < 3; e++) {
      const Pt *u = v[e], *w = v[(e + 1) % 3];
      double mx = 0.5 * (u->x + w->x), my = 0.5 * (u->y + w->y);
      double g = 0.5 * ((Z1 - u->H) + (Z1 - w->H));
      double wq = A / 3.0;
      s->x += wq * mx;
      s->y += wq * my;
      s->xg += wq * mx * g;
      s->yg += wq * my * g;
      s->zg += wq * g * (top - 0.5 * g);
    }
  }
}

/* Moments of the fluid part of one box: footprint rectangle
 * [a0/2, a1/2] x [b0/2, b1/2] of lattice square (I, J), heights [Z0, Z1].
 * Coordinates of the results: xi, eta local to the square, Z - zb. */
typedef struct {
  double vol, mx, my, mz;
  double fa[6], f1[6], f2[6];  /* faces xlo, xhi, ylo, yhi, zlo, zhi */
  double eba, ebx, eby, ebz;   /* physical EB area per dx*dy and its moments */
  double nv[3], rv[3];
  int flag;
} BoxMom;

/* One vertical face profile: the side of the rectangle at xi = c (axis 0) or
 * eta = c (axis 1), from s0 to s1 (half-lattice units).  Accumulates the
 * fluid area, int s * g, int Z. */
static void face_profile(const double Hq[3][3], int axis, int c2, int s0, int s1, double Z0, double Z1,
                         double zb, double *fa, double *fs, double *fz) {
  double A = 0, S = 0, Zm = 0;
  for (int q = s0; q < s1; q++) {
    double sa = 0.5 * q, sb = 0.5 * (q + 1);
    double Ha = axis == 0 ? Hq[c2][q] : Hq[q][c2];
    double Hb = axis == 0 ? Hq[c2][q + 1] : Hq[q + 1][c2];
    /* split [sa, sb] where H crosses Z0 and Z1 */
    double ts[4];
    int nt = 0;
    ts[nt++] = 0.0;
    double lv[2] = {Z0, Z1};
    double tc[2];
    int nc = 0;
    for (int l = 0; l < 2; l++) {
      if ((Ha < lv[l]) != (Hb < lv[l])) {
        double t = (lv[l] - Ha) / (Hb - Ha);
        tc[nc++] = t;
      }
    }
    if (nc == 2 && tc[0] > tc[1]) { double tmp = tc[0]; tc[0] = tc[1]; tc[1] = tmp; }
    for (int l = 0; l < nc; l++) ts[nt++] = tc[l];
    ts[nt++] = 1.0;
    for (int r = 0; r + 1 < nt; r++) {
      double t0 = ts[r], t1 = ts[r + 1];
      if (!(t1 > t0)) continue;
      double tm = 0.5 * (t0 + t1);
      double Hm = Ha + tm * (Hb - Ha);
      double len = (t1 - t0) * (sb - sa);
      double tt[3] = {t0, tm, t1};
      double wt[3] = {1.0 / 6.0, 4.0 / 6.0, 1.0 / 6.0};
      if (Hm < Z0) {
        /* full height: constant integrand, integrated exactly */
        double g = Z1 - Z0;
        double s0 = sa + t0 * (sb - sa), s1 = sa + t1 * (sb - sa);
        A += len * g;
        S += g * 0.5 * (s0 + s1) * len;
        Zm += len * 0.5 * ((Z1 - zb) * (Z1 - zb) - (Z0 - zb) * (Z0 - zb));
      } else if (Hm < Z1) {
        for (int e = 0; e < 3; e++) {
          double s = sa + tt[e] * (sb - sa);
          double H = Ha + tt[e] * (Hb - Ha);
          double g = Z1 - H;
          A += len * wt[e] * g;
          S += len * wt[e] * s * g;
          /* z-moment of the fluid column [H, Z1] about zb: g (Z1 - zb - g/2) */
          Zm += len * wt[e] * g * ((Z1 - zb) - 0.5 * g);
        }
      }
    }
  }
  *fa += A; *fs += S; *fz += Zm;
}

static int box_flag(const double Hq[3][3], int a0, int a1, int b0, int b1, double Z0, double Z1) {
  double mn = 1e300, mx = -1e300;
  for (int a = a0; a <= a1; a++)
    for (int b = b0; b <= b1; b++) {
      if (Hq[a][b] < mn) mn = Hq[a][b];
      if (Hq[a][b] > mx) mx = Hq[a][b];
    }
  if (mn >= Z1) return ORC_COVERED;
  if (mx < Z0) return ORC_REGULAR;
  return ORC_CUT;
}

static void box_moments(const double Hq[3][3], int a0, int a1, int b0, int b1, double Z0, double Z1,
                        double zb, double sx, double sy, BoxMom *m) {
  memset(m, 0, sizeof(*m));
  m->flag = box_flag(Hq, a0, a1, b0, b1, Z0, Z1);
  /* vertical faces */
  face_profile(Hq, 0, a0, b0, b1, Z0, Z1, zb, &m->fa[0], &m->f1[0], &m->f2[0]);
  face_profile(Hq, 0, a1, b0, b1, Z0, Z1, zb, &m->fa[1], &m->f1[1], &m->f2[1]);
  face_profile(Hq, 1, b0, a0, a1, Z0, Z1, zb, &m->fa[2], &m->f1[2], &m->f2[2]);
  face_profile(Hq, 1, b1, a0, a1, Z0, Z1, zb, &m->fa[3], &m->f1[3], &m->f2[3]);
  /* the two triangles of the square */
  Pt T[2][3] = {{{0, 0, Hq[0][0]}, {1, 0, Hq[2][0]}, {1, 1, Hq[2][2]}},
                {{0, 0, Hq[0][0]}, {1, 1, Hq[2][2]}, {0, 1, Hq[0][2]}}};
  double gx[2] = {Hq[2][0] - Hq[0][0], Hq[2][2] - Hq[0][2]};
  double gy[2] = {Hq[2][2] - Hq[2][0], Hq[0][2] - Hq[0][0]};
  for (int t = 0; t < 2; t++) {
    Pt b1p[8], b2p[8];
    int n = 3;
    memcpy(b1p, T[t], sizeof(T[t]));
    n = clip_coord(b1p, n, 0, 0.5 * a1, 1.0, b2p);
    n = clip_coord(b2p, n, 0, 0.5 * a0, -1.0, b1p);
    n = clip_coord(b1p, n, 1, 0.5 * b1, 1.0, b2p);
    n = clip_coord(b2p, n, 1, 0.5 * b0, -1.0, b1p);
    if (n < 3) continue;
    /* heights from the half lattice */
    for (int v = 0; v < n; v++) b1p[v].H = Hq[(int)(2.0 * b1p[v].x)][(int)(2.0 * b1p[v].y)];
    Pt A[12], B[12], Bt[12], U[12];
    int nA = clip_level(b1p, n, Z0, 1, A);
    int nB0 = clip_level(b1p, n, Z0, 0, Bt);
    int nB = clip_level(Bt, nB0, Z1, 1, B);
    int nU = clip_level(b1p, n, Z1, 1, U);
    PolyInt sA, sB, sU;
    poly_integrals(A, nA, zb, Z1, &sA);
    poly_integrals(B, nB, zb, Z1, &sB);
    poly_integrals(U, nU, zb, Z1, &sU);
    double hgt = Z1 - Z0;
    /* region A: H < Z0, full height */
    m->vol += hgt * sA.a;
    m->mx += hgt * sA.x;
    m->my += hgt * sA.y;
    m->mz += 0.5 * ((Z1 - zb) * (Z1 - zb) - (Z0 - zb) * (Z0 - zb)) * sA.a;
    /* region B: Z0 <= H < Z1, height Z1 - H */
    m->vol += sB.g;
    m->mx += sB.xg;
    m->my += sB.yg;
    m->mz += sB.zg;
    /* horizontal faces: bottom open where H < Z0, top open where H < Z1 */
    m->fa[4] += sA.a; m->f1[4] += sA.x; m->f2[4] += sA.y;
    m->fa[5] += sU.a; m->f1[5] += sU.x; m->f2[5] += sU.y;
    /* EB facet: the plane over region B */
    if (sB.a > 0.0) {
      double hx = sx * gx[t], hy = sy * gy[t];
      double el = sqrt(1.0 + hx * hx + hy * hy);
      double ar = sB.a * el;
      m->eba += ar;
      m->ebx += el * sB.x;
      m->eby += el * sB.y;
      m->ebz += el * ((Z1 - zb) * sB.a - sB.g);
      m->nv[0] += -hx * sB.a; m->nv[1] += -hy * sB.a; m->nv[2] += sB.a;
      m->rv[0] += -gx[t] * sB.a; m->rv[1] += -gy[t] * sB.a; m->rv[2] += sB.a;
    }
  }
}

/* Accumulator for a CV made of one or two half-cells, in CV-local
 * coordinates (origin at the CV centre). */
typedef struct {
  double vol, m[3];
  double fa[3], f1[3], f2[3];   /* LOW faces only: x, y, z */
  double eba, eb[3], nv[3], rv[3];
  int ncov, nreg, nbox;
} CvAcc;

/* Add a box, shifting its xi, eta, Z coordinates by (ox, oy, oz) into CV
 * coordinates; lowface[d] selects which face of the box (0: low side,
 * 1: high side, -1: none) is part of the CV's low d-face. */
static void cv_add(CvAcc *c, const BoxMom *b, double ox, double oy, double oz, const int lowface[3]) {
  c->nbox++;
  if (b->flag == ORC_COVERED) c->ncov++;
  if (b->flag == ORC_REGULAR) c->nreg++;
  c->vol += b->vol;
  c->m[0] += b->mx + ox * b->vol;
  c->m[1] += b->my + oy * b->vol;
  c->m[2] += b->mz + oz * b->vol;
  /* x faces: transverse (eta, Z); y faces: (xi, Z); z faces: (xi, eta) */
  for (int d = 0; d < 3; d++) {
    if (lowface[d] < 0) continue;
    int f = 2 * d + lowface[d];
    double t1o = d == 0 ? oy : ox;
    double t2o = d == 2 ? oy : oz;
    c->fa[d] += b->fa[f];
    c->f1[d] += b->f1[f] + t1o * b->fa[f];
    c->f2[d] += b->f2[f] + t2o * b->fa[f];
  }
  c->eba += b->eba;
  c->eb[0] += b->ebx + ox * b->eba;
  c->eb[1] += b->eby + oy * b->eba;
  c->eb[2] += b->ebz + oz * b->eba;
  for (int d = 0; d < 3; d++) { c->nv[d] += b->nv[d]; c->rv[d] += b->rv[d]; }
}

static void cv_store(const CvAcc *c, OrcGeom *G, long n, long id) {
  int flag = (c->ncov == c->nbox) ? ORC_COVERED : (c->nreg == c->nbox) ? ORC_REGULAR : ORC_CUT;
  G->flag[id] = (uint8_t)flag;
  G->alpha[id] = c->vol;
  for (int d = 0; d < 3; d++) {
    G->cent[d * n + id] = c->vol > 0 ? c->m[d] / c->vol : 0.0;
    G->beta[d * n + id] = c->fa[d];
    G->fcent[(2 * d) * n + id] = c->fa[d] > 0 ? c->f1[d] / c->fa[d] : 0.0;
    G->fcent[(2 * d + 1) * n + id] = c->fa[d] > 0 ? c->f2[d] / c->fa[d] : 0.0;
    G->ebc[d * n + id] = c->eba > 0 ? c->eb[d] / c->eba : 0.0;
    G->ebv[d * n + id] = c->rv[d];
  }
  G->aeb[id] = c->eba;
  double nn = sqrt(c->nv[0] * c->nv[0] + c->nv[1] * c->nv[1] + c->nv[2] * c->nv[2]);
  for (int d = 0; d < 3; d++) G->nrm[d * n + id] = nn > 0 ? c->nv[d] / nn : 0.0;
}

/* Geometry of grid g over the window (Sec. 3.2).  c-grid CVs are single
 * cells; a u-grid CV (i,j,k) is the right half of cell i-1 plus the left half
 * of cell i; v likewise in y; a w-grid CV (i,j,k) is the top half of cell k-1
 * plus the bottom half of cell k (only one half at the walls k = 0, nz).
 * Areas and volumes add; the EB normal and centroid are area weighted. */
int orc_geometry(const OrcDomain *D, int g, OrcGeom *G) {
  long n = ncv(D, g);
  int nzg = nzg_of(D, g);
  double sx = D->dz / D->dx, sy = D->dz / D->dy;
#pragma omp parallel for schedule(dynamic, 1)
  for (int k = 0; k < nzg; k++) {
    for (int lj = 0; lj < D->WY; lj++) {
      for (int li = 0; li < D->WX; li++) {
        int gi = D->x0 + li, gj = D->y0 + lj;
        long id = (long)li + (long)D->WX * ((long)lj + (long)D->WY * k);
        CvAcc c;
        memset(&c, 0, sizeof(c));
        double Hq[3][3];
        BoxMom b;
        if (g == GC) {
          half_lattice(D, gi, gj, Hq);
          box_moments(Hq, 0, 2, 0, 2, k, k + 1, k, sx, sy, &b);
          int lf[3] = {0, 0, 0};
          cv_add(&c, &b, -0.5, -0.5, -0.5, lf);
        } else if (g == GU) {
          int lf1[3] = {0, 0, 0}, lf2[3] = {-1, 0, 0};
          half_lattice(D, gi - 1, gj, Hq);
          box_moments(Hq, 1, 2, 0, 2, k, k + 1, k, sx, sy, &b);
          cv_add(&c, &b, -1.0, -0.5, -0.5, lf1);
          half_lattice(D, gi, gj, Hq);
          box_moments(Hq, 0, 1, 0, 2, k, k + 1, k, sx, sy, &b);
          cv_add(&c, &b, 0.0, -0.5, -0.5, lf2);
        } else if (g == GV) {
          int lf1[3] = {0, 0, 0}, lf2[3] = {0, -1, 0};
          half_lattice(D, gi, gj - 1, Hq);
          box_moments(Hq, 0, 2, 1, 2, k, k + 1, k, sx, sy, &b);
          cv_add(&c, &b, -0.5, -1.0, -0.5, lf1);
          half_lattice(D, gi, gj, Hq);
          box_moments(Hq, 0, 2, 0, 1, k, k + 1, k, sx, sy, &b);
          cv_add(&c, &b, -0.5, 0.0, -0.5, lf2);
        } else {
          half_lattice(D, gi, gj, Hq);
          if (k >= 1) {
            int lf1[3] = {0, 0, 0};
            box_moments(Hq, 0, 2, 0, 2, k - 0.5, k, k, sx, sy, &b);
            cv_add(&c, &b, -0.5, -0.5, 0.0, lf1);
          }
          if (k <= D->nz - 1) {
            int lf2[3] = {0, 0, -1};
            box_moments(Hq, 0, 2, 0, 2, k, k + 0.5, k, sx, sy, &b);
            cv_add(&c, &b, -0.5, -0.5, 0.0, lf2);
          }
        }
        cv_store(&c, G, n, id);
      }
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* 2. Fluxes and the cut-cell update (Sec. 3.1 and 4.1)                       */
/* ------------------------------------------------------------------------- */

typedef struct {
  double *f[5];   /* rho, rho*theta (c grid), rho*u (u), rho*v (v), rho*w (w) */
} OrcState;

static const int FIELD_GRID[5] = {GC, GC, GU, GV, GW};

/* Is CV (gi,gj,k) of grid g inside the domain, in the window and not covered?
 * These are the CVs whose values a flux stencil may use. */
static long avail(const OrcDomain *D, const OrcGeom *G, int g, int gi, int gj, int k) {
  long id = loc(D, g, gi, gj, k);
  if (id < 0) return -1;
  if (!(G[g].alpha[id] > 0.0)) return -1;
  return id;
}

/* Prognostic CVs: every non-covered CV except the two wall levels of w. */
static int prognostic(const OrcDomain *D, int g, int k) {
  return !(g == GW && (k == 0 || k == D->nz));
}

/* Momentum of a CV as it enters a mass flux: zero where the CV is covered,
 * absent, or a wall level of w. */
static double mom(const OrcDomain *D, const OrcGeom *G, const OrcState *U, int g, int gi, int gj, int k) {
  long id = avail(D, G, g, gi, gj, k);
  if (id < 0) return 0.0;
  if (g == GW && (k == 0 || k == D->nz)) return 0.0;
  return U->f[g == GU ? 2 : g == GV ? 3 : 4][id];
}

/* Advected value of a CV: theta on c, the velocity component on u, v, w.
 * Face velocities divide the momentum by the mean density of the non-covered
 * cells beside the face; w is zero on the wall levels. */
static double advected(const OrcDomain *D, const OrcGeom *G, const OrcState *U, int g, int gi, int gj, int k,
                       long id) {
  if (g == GC) return U->f[1][id] / U->f[0][id];
  if (g == GW && (k == 0 || k == D->nz)) return 0.0;
  int di = g == GU, dj = g == GV, dk = g == GW;
  long a = avail(D, G, GC, gi - di, gj - dj, k - dk);
  long b = avail(D, G, GC, gi, gj, k);
  double rb;
  if (a >= 0 && b >= 0) rb = 0.5 * (U->f[0][a] + U->f[0][b]);
  else if (a >= 0) rb = U->f[0][a];
  else if (b >= 0) rb = U->f[0][b];
  else return 0.0;
  return U->f[g == GU ? 2 : g == GV ? 3 : 4][id] / rb;
}

/* Mass flux through the low d-face of CV (gi,gj,k) of grid g. */
static double mass_flux(const OrcDomain *D, const OrcGeom *G, const OrcState *U, int g, int d, int gi, int gj,
                        int k) {
  if (g == GC) {
    if (d == 0) return mom(D, G, U, GU, gi, gj, k);
    if (d == 1) return mom(D, G, U, GV, gi, gj, k);
    return mom(D, G, U, GW, gi, gj, k);
  }
  /* the momentum grid that carries direction d */
  int mg = d == 0 ? GU : d == 1 ? GV : GW;
  if (mg == g) {
    /* face at the centre of the cell below, between CVs p - e_d and p */
    int di = d == 0, dj = d == 1, dk = d == 2;
    return 0.5 * (mom(D, G, U, mg, gi - di, gj - dj, k - dk) + mom(D, G, U, mg, gi, gj, k));
  }
  /* edge face: average the two momenta of grid mg straddling it, offset
   * along the staggering axis of g */
  int si = g == GU, sj = g == GV, sk = g == GW;
  return 0.5 * (mom(D, G, U, mg, gi - si, gj - sj, k - sk) + mom(D, G, U, mg, gi, gj, k));
}

/* Provisional flux of advected value phi through the low d-face of CV p:
 * third-order upwind, i.e. fourth-order centred plus hyperviscosity, falling
 * back to second-order centred when the far upstream CV is covered or beyond
 * a wall (Sec. 4.1).  Returns 0 for a closed face. */
static void face_flux(const OrcDomain *D, const OrcGeom *G, const OrcState *U, int g, int d, int gi, int gj,
                      int k, double *Fm, double *Fphi) {
  *Fm = 0.0;
  *Fphi = 0.0;
  long p = loc(D, g, gi, gj, k);
  if (p < 0) return;
  if (!(G[g].beta[(long)d * ncv(D, g) + p] > 0.0)) return;
  int di = d == 0, dj = d == 1, dk = d == 2;
  long L = avail(D, G, g, gi - di, gj - dj, k - dk);
  long R = avail(D, G, g, gi, gj, k);
  if (L < 0 || R < 0) return;
  double m = mass_flux(D, G, U, g, d, gi, gj, k);
  *Fm = m;
  if (m == 0.0) return;
  double pL = advected(D, G, U, g, gi - di, gj - dj, k - dk, L);
  double pR = advected(D, G, U, g, gi, gj, k, R);
  double val;
  if (m > 0.0) {
    long F = avail(D, G, g, gi - 2 * di, gj - 2 * dj, k - 2 * dk);
    if (F >= 0) {
      double pF = advected(D, G, U, g, gi - 2 * di, gj - 2 * dj, k - 2 * dk, F);
      val = (-pF + 5.0 * pL + 2.0 * pR) / 6.0;
    } else {
      val = 0.5 * (pL + pR);
    }
  } else {
    long F = avail(D, G, g, gi + di, gj + dj, k + dk);
    if (F >= 0) {
      double pF = advected(D, G, U, g, gi + di, gj + dj, k + dk, F);
      val = (2.0 * pL + 5.0 * pR - pF) / 6.0;
    } else {
      val = 0.5 * (pL + pR);
    }
  }
  *Fphi = m * val;
}

/* Is the low d-face of CV (gi,gj,k) of grid g a usable neighbour face for the
 * centroid interpolation: inside the domain (w-grid faces of the two wall
 * levels excluded) and open? */
static long face_open(const OrcDomain *D, const OrcGeom *G, int g, int d, int gi, int gj, int k) {
  if (g == GW && d != 2 && (k < 1 || k > D->nz - 1)) return -1;
  long p = loc(D, g, gi, gj, k);
  if (p < 0) return -1;
  if (!(G[g].beta[(long)d * ncv(D, g) + p] > 0.0)) return -1;
  return p;
}

/* Centroid flux of the low d-face of CV p: bilinear interpolation of the
 * provisional fluxes of the face and its neighbours toward the face centroid
 * (Sec. 4.1, flux interpolation).  A transverse offset is dropped when a
 * neighbour face it needs is closed or outside the domain. */
static double centroid_flux(const OrcDomain *D, const OrcGeom *G, int g, int d, int gi, int gj, int k, long p,
                            const double *Fh) {
  long n = ncv(D, g);
  int ta = d == 0 ? 1 : 0, tb = d == 2 ? 1 : 2;
  double ga = G[g].fcent[(2 * d) * n + p], gb = G[g].fcent[(2 * d + 1) * n + p];
  if (ga == 0.0 && gb == 0.0) return Fh[p];
  int sa = ga >= 0.0 ? 1 : -1, sb = gb >= 0.0 ? 1 : -1;
  int ea[3] = {0, 0, 0}, eb[3] = {0, 0, 0};
  ea[ta] = sa;
  eb[tb] = sb;
  long pa = -1, pb = -1, pab = -1;
  if (ga != 0.0) pa = face_open(D, G, g, d, gi + ea[0], gj + ea[1], k + ea[2]);
  if (gb != 0.0) pb = face_open(D, G, g, d, gi + eb[0], gj + eb[1], k + eb[2]);
  if (ga != 0.0 && gb != 0.0)
    pab = face_open(D, G, g, d, gi + ea[0] + eb[0], gj + ea[1] + eb[1], k + ea[2] + eb[2]);
  int za = ga != 0.0 && (pa < 0 || (gb != 0.0 && pab < 0));
  int zb = gb != 0.0 && (pb < 0 || (ga != 0.0 && pab < 0));
  double wa = za ? 0.0 : fabs(ga), wb = zb ? 0.0 : fabs(gb);
  double F = (1.0 - wa) * (1.0 - wb) * Fh[p];
  if (wa > 0.0) F += wa * (1.0 - wb) * Fh[pa];
  if (wb > 0.0) F += wb * (1.0 - wa) * Fh[pb];
  if (wa > 0.0 && wb > 0.0) F += wa * wb * Fh[pab];
  return F;
}

/* Flux divergence dU of every prognostic non-covered CV (Eqs. update-cc and
 * update-fc, with zero flux through the EB and the domain walls); zero
 * elsewhere. */
int orc_flux_div(const OrcDomain *D, const OrcGeom *G, const OrcState *U, OrcState *dU) {
  double dd[3] = {D->dx, D->dy, D->dz};
  for (int g = 0; g < 4; g++) {
    long n = ncv(D, g);
    int nzg = nzg_of(D, g);
    int nf = g == GC ? 2 : 1;  /* c grid: mass and rho*theta */
    double *Fh = malloc(sizeof(double) * (size_t)n * 3 * 2);
    double *Fc = malloc(sizeof(double) * (size_t)n * 3 * 2);
    /* provisional fluxes */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nzg; k++)
      for (int lj = 0; lj < D->WY; lj++)
        for (int li = 0; li < D->WX; li++) {
          long id = (long)li + (long)D->WX * ((long)lj + (long)D->WY * k);
          for (int d = 0; d < 3; d++) {
            double fm, fp;
            face_flux(D, G, U, g, d, D->x0 + li, D->y0 + lj, k, &fm, &fp);
            Fh[(0 * 3 + d) * n + id] = fm;
            Fh[(1 * 3 + d) * n + id] = fp;
          }
        }
    /* centroid fluxes */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nzg; k++)
      for (int lj = 0; lj < D->WY; lj++)
        for (int li = 0; li < D->WX; li++) {
          long id = (long)li + (long)D->WX * ((long)lj + (long)D->WY * k);
          for (int d = 0; d < 3; d++)
            for (int q = 0; q < 2; q++) {
              double *src = Fh + (q * 3 + d) * n;
              double F = 0.0;
              if (G[g].beta[(long)d * n + id] > 0.0)
                F = centroid_flux(D, G, g, d, D->x0 + li, D->y0 + lj, k, id, src);
              Fc[(q * 3 + d) * n + id] = F;
            }
        }
    /* divergence */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nzg; k++)
      for (int lj = 0; lj < D->WY; lj++)
        for (int li = 0; li < D->WX; li++) {
          long id = (long)li + (long)D->WX * ((long)lj + (long)D->WY * k);
          int gi = D->x0 + li, gj = D->y0 + lj;
          for (int q = 0; q < nf; q++) {
            int fld = g == GC ? q : (g + 1);
            double out = 0.0;
            if (G[g].alpha[id] > 0.0 && prognostic(D, g, k)) {
              double s = 0.0;
              for (int d = 0; d < 3; d++) {
                int di = d == 0, dj = d == 1, dk = d == 2;
                double lo = G[g].beta[(long)d * n + id] * Fc[((g == GC ? q : 1) * 3 + d) * n + id];
                double hi = 0.0;
                long up = loc(D, g, gi + di, gj + dj, k + dk);
                if (up >= 0) hi = G[g].beta[(long)d * n + up] * Fc[((g == GC ? q : 1) * 3 + d) * n + up];
                s += (hi - lo) / dd[d];
              }
              out = -s / G[g].alpha[id];
            }
            dU->f[fld][id] = out;
          }
        }
    free(Fh);
    free(Fc);
    (void)nf;
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* 3. Weighted state redistribution (Sec. 5.1)                                */
/* ------------------------------------------------------------------------- */
/*
 * Neighbourhood code of a small CV (shared with the GPU library's export
 * format, which is why it is spelled out): axes a1, a2, a3 ordered by
 * decreasing |n_d| of the unit EB normal (two components count as equal when
 * they differ by at most 1e-12; ties go x before y before z), signs
 * s_d = sign(n_d) with sign(0) = +1, where a component within 1e-12 of zero
 * counts as zero, and the growth level L (1: two cells,
 * 2: 2 x 2, 3: 2 x 2 x 2).  perm index p over the orderings
 * (xyz, xzy, yxz, yzx, zxy, zyx), sign bits sx | sy<<1 | sz<<2 (bit set =
 * negative);  code = 1 + (p*8 + signbits)*3 + (L-1), and 0 for CVs that are
 * not small.
 */
static const int PERMS[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

static void axis_order(const double n[3], int ax[3]) {
  const double tol = 1e-12;
  double a[3] = {fabs(n[0]), fabs(n[1]), fabs(n[2])};
  /* a1: the lowest-index axis not beaten by another by more than tol */
  int first = -1;
  for (int d = 0; d < 3 && first < 0; d++) {
    int ok = 1;
    for (int e = 0; e < 3; e++)
      if (e != d && a[e] > a[d] + tol) ok = 0;
    if (ok) first = d;
  }
  int r0 = -1, r1 = -1;
  for (int d = 0; d < 3; d++)
    if (d != first) { if (r0 < 0) r0 = d; else r1 = d; }
  ax[0] = first;
  if (a[r1] > a[r0] + tol) { ax[1] = r1; ax[2] = r0; }
  else { ax[1] = r0; ax[2] = r1; }
}

/* Candidate offsets of a neighbourhood with axes ax, signs s, in growth
 * order; returns how many candidates level L holds (2, 4 or 8). */
static int nbhd_offsets(const int ax[3], const int s[3], int L, int off[8][3]) {
  int cnt = L == 1 ? 2 : L == 2 ? 4 : 8;
  for (int c = 0; c < 8; c++) {
    off[c][0] = off[c][1] = off[c][2] = 0;
    int b1 = c & 1, b2 = (c >> 1) & 1, b3 = (c >> 2) & 1;
    if (b1) off[c][ax[0]] += s[ax[0]];
    if (b2) off[c][ax[1]] += s[ax[1]];
    if (b3) off[c][ax[2]] += s[ax[2]];
  }
  return cnt;
}

static void decode(int code, int ax[3], int s[3], int *L) {
  int c = code - 1;
  *L = c % 3 + 1;
  c /= 3;
  int sb = c % 8, p = c / 8;
  for (int d = 0; d < 3; d++) { ax[d] = PERMS[p][d]; s[d] = ((sb >> d) & 1) ? -1 : 1; }
}

static int perm_index(const int ax[3]) {
  for (int p = 0; p < 6; p++)
    if (PERMS[p][0] == ax[0] && PERMS[p][1] == ax[1] && PERMS[p][2] == ax[2]) return p;
  return 0;
}

/* CVs that take part in redistribution: non-covered and prognostic. */
static long active(const OrcDomain *D, const OrcGeom *Gg, int g, int gi, int gj, int k) {
  long id = loc(D, g, gi, gj, k);
  if (id < 0) return -1;
  if (!(Gg->alpha[id] > 0.0)) return -1;
  if (!prognostic(D, g, k)) return -1;
  return id;
}

/* Members of the neighbourhood of CV (gi,gj,k) (code != 0): window ids and
 * offsets of the active candidates; returns the count (>= 1, self first). */
static int members(const OrcDomain *D, const OrcGeom *Gg, int g, int gi, int gj, int k, int code, long *mid,
                   int moff[8][3]) {
  int ax[3], s[3], L;
  decode(code, ax, s, &L);
  int off[8][3];
  int cnt = nbhd_offsets(ax, s, L, off);
  int m = 0;
  for (int c = 0; c < cnt; c++) {
    long id = active(D, Gg, g, gi + off[c][0], gj + off[c][1], k + off[c][2]);
    if (id < 0) continue;
    mid[m] = id;
    moff[m][0] = off[c][0]; moff[m][1] = off[c][1]; moff[m][2] = off[c][2];
    m++;
  }
  return m;
}

/* x - xhat_r for a point x given relative to r's centre, formed as
 * sum_m w_m (x - x_m) over the members of M_r with the weights of Eq.
 * centroid (they sum to one): no cancellation when xhat_r lies close to one
 * member, as it does for a tiny cell merged into one large neighbour. */
static void from_xhat(const OrcDomain *D, int g, const OrcGeom *Gg, const OrcWsrd *W, int gi, int gj, int k, long r,
                      const double x[3], double e[3]) {
  long n = ncv(D, g);
  e[0] = e[1] = e[2] = 0.0;
  long mid[8];
  int moff[8][3];
  int nm = W->code[r] ? members(D, Gg, g, gi, gj, k, W->code[r], mid, moff) : 1;
  if (!W->code[r]) { mid[0] = r; moff[0][0] = moff[0][1] = moff[0][2] = 0; }
  for (int q = 0; q < nm; q++) {
    double wq = q == 0 ? W->omega[r] * Gg->alpha[r] / W->vhat[r]
                       : W->kappa[r] * Gg->alpha[mid[q]] / W->nnb[mid[q]] / W->vhat[r];
    for (int a = 0; a < 3; a++) e[a] += wq * (x[a] - (moff[q][a] + Gg->cent[a * n + mid[q]]));
  }
}

/* Set-up of the redistribution tables of grid g: small CVs, their merging
 * neighbourhoods M, N, kappa (Eq. kappa, clamped to 1), omega (Eq. omega),
 * the weighted volume (Eq. nbhd_vol) and centroid (Eq. centroid). */
int orc_wsrd_setup(const OrcDomain *D, int g, const OrcGeom *Gg, double vt, OrcWsrd *W) {
  long n = ncv(D, g);
  int nzg = nzg_of(D, g);
  /* neighbourhoods and kappa */
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nzg; k++)
    for (int lj = 0; lj < D->WY; lj++)
      for (int li = 0; li < D->WX; li++) {
        long id = (long)li + (long)D->WX * ((long)lj + (long)D->WY * k);
        int gi = D->x0 + li, gj = D->y0 + lj;
        W->code[id] = 0;
        W->kappa[id] = 0.0;
        if (active(D, Gg, g, gi, gj, k) < 0) continue;
        double V = Gg->alpha[id];
        if (!(V < vt)) continue;
        double nv[3] = {Gg->nrm[id], Gg->nrm[n + id], Gg->nrm[2 * n + id]};
        int ax[3], s[3], sb = 0;
        axis_order(nv, ax);
        for (int d = 0; d < 3; d++) { s[d] = nv[d] < -1e-12 ? -1 : 1; if (s[d] < 0) sb |= 1 << d; }
        int L;
        double sum = 0.0;
        for (L = 1; L <= 3; L++) {
          int off[8][3];
          int cnt = nbhd_offsets(ax, s, L, off);
          sum = 0.0;
          for (int c = 1; c < cnt; c++) {
            long m = active(D, Gg, g, gi + off[c][0], gj + off[c][1], k + off[c][2]);
            if (m >= 0) sum += Gg->alpha[m];
          }
          if (!(V + sum < vt)) break;
        }
        if (L > 3) L = 3;
        W->code[id] = (uint8_t)(1 + (perm_index(ax) * 8 + sb) * 3 + (L - 1));
        double kap = sum > 0.0 ? (vt - V) / sum : 0.0;
        W->kappa[id] = kap > 1.0 ? 1.0 : kap;
      }
  /* N and omega, gathered over the 26 neighbours whose neighbourhoods may
   * contain the CV */
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nzg; k++)
    for (int lj = 0; lj < D->WY; lj++)
      for (int li = 0; li < D->WX; li++) {
        long id = (long)li + (long)D->WX * ((long)lj + (long)D->WY * k);
        int gi = D->x0 + li, gj = D->y0 + lj;
        W->nnb[id] = 0;
        W->omega[id] = 0.0;
        if (active(D, Gg, g, gi, gj, k) < 0) continue;
        int N = 1;
        double ks = 0.0;
        for (int dk = -1; dk <= 1; dk++)
          for (int dj = -1; dj <= 1; dj++)
            for (int di = -1; di <= 1; di++) {
              if (!di && !dj && !dk) continue;
              long r = active(D, Gg, g, gi + di, gj + dj, k + dk);
              if (r < 0 || W->code[r] == 0) continue;
              long mid[8];
              int moff[8][3];
              int nm = members(D, Gg, g, gi + di, gj + dj, k + dk, W->code[r], mid, moff);
              for (int q = 1; q < nm; q++)
                if (moff[q][0] == -di && moff[q][1] == -dj && moff[q][2] == -dk) {
                  N++;
                  ks += W->kappa[r];
                }
            }
        W->nnb[id] = N;
        W->omega[id] = 1.0 - ks / N;
      }
  /* weighted volume and centroid */
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nzg; k++)
    for (int lj = 0; lj < D->WY; lj++)
      for (int li = 0; li < D->WX; li++) {
        long id = (long)li + (long)D->WX * ((long)lj + (long)D->WY * k);
        int gi = D->x0 + li, gj = D->y0 + lj;
        W->vhat[id] = 0.0;
        W->xhat[id] = W->xhat[n + id] = W->xhat[2 * n + id] = 0.0;
        if (active(D, Gg, g, gi, gj, k) < 0) continue;
        double V = Gg->alpha[id];
        double vh = W->omega[id] * V;
        double xs[3];
        for (int d = 0; d < 3; d++) xs[d] = W->omega[id] * V * Gg->cent[d * n + id];
        if (W->code[id]) {
          long mid[8];
          int moff[8][3];
          int nm = members(D, Gg, g, gi, gj, k, W->code[id], mid, moff);
          for (int q = 1; q < nm; q++) {
            double w = W->kappa[id] * Gg->alpha[mid[q]] / W->nnb[mid[q]];
            vh += w;
            for (int d = 0; d < 3; d++) xs[d] += w * (moff[q][d] + Gg->cent[d * n + mid[q]]);
          }
        }
        W->vhat[id] = vh;
        for (int d = 0; d < 3; d++) W->xhat[d * n + id] = xs[d] / vh;
      }
  return 0;
}

/* Neighbourhood averages are kept in the pivoted deviation form
 * Qhat_r = Uhat[piv_r] + D_r,  D_r = sum_{m != p} w_m (Uhat_m - Uhat_p),
 * which equals Eq. qhat_omega because the weights w sum to one; the pivot p
 * is the first member with V >= V_target, else the first largest member.
 * Non-small CVs have piv = itself and D = 0 (their neighbourhood is
 * themselves).  Every difference of two averages is then formed as
 * (Uhat[piv_a] - Uhat[piv_b]) + (D_a - D_b): for a tiny cell merged with one
 * large neighbour, Qhat_r lies within ~alpha of that neighbour's value and
 * the difference is kept to full relative accuracy. */
typedef struct { const double *Uh; const long *piv; const double *D; } QhatForm;

static double qdiff(const QhatForm *Q, long a, long b) {
  return (Q->Uh[Q->piv[a]] - Q->Uh[Q->piv[b]]) + (Q->D[a] - Q->D[b]);
}

/* Least-squares gradient of Qhat for small CV r (Sec. 5.1): fit over the
 * non-covered CVs of the 3x3x3 box around r, each Qhat placed at its
 * neighbourhood centroid; an axis whose centroid spread is below half a cell
 * is widened to 5; the gradient is zero when the box still lacks spread, has
 * fewer than 4 points, or the normal matrix is near singular.  Then the
 * Barth-Jespersen-style limiter: the reconstruction at the centroids of the
 * neighbourhood's members may not leave [Qmin, Qmax] of the stencil and r.
 * Returns the limiter factor. */
static double lsq_gradient(const OrcDomain *D, int g, const OrcGeom *Gg, const OrcWsrd *W, const QhatForm *Q,
                           int gi, int gj, int k, long r, double sig[3]) {
  long n = ncv(D, g);
  double xr[3] = {W->xhat[r], W->xhat[n + r], W->xhat[2 * n + r]};
  int w[3] = {1, 1, 1};
  sig[0] = sig[1] = sig[2] = 0.0;
  double M[3][3], b[3];
  double bmax = 0.0, bmin = 0.0;   /* Qmax - Qhat_r and Qmin - Qhat_r */
  int cnt = 0;
  for (int pass = 0; pass < 2; pass++) {
    double spread[3] = {0, 0, 0};
    memset(M, 0, sizeof(M));
    b[0] = b[1] = b[2] = 0.0;
    bmax = bmin = 0.0;
    cnt = 0;
    for (int dk = -w[2]; dk <= w[2]; dk++)
      for (int dj = -w[1]; dj <= w[1]; dj++)
        for (int di = -w[0]; di <= w[0]; di++) {
          if (!di && !dj && !dk) continue;
          long m = active(D, Gg, g, gi + di, gj + dj, k + dk);
          if (m < 0) continue;
          double dv[3] = {di + W->xhat[m] - xr[0], dj + W->xhat[n + m] - xr[1], dk + W->xhat[2 * n + m] - xr[2]};
          double dq = qdiff(Q, m, r);
          for (int a = 0; a < 3; a++) {
            if (fabs(dv[a]) > spread[a]) spread[a] = fabs(dv[a]);
            b[a] += dv[a] * dq;
            for (int c = 0; c < 3; c++) M[a][c] += dv[a] * dv[c];
          }
          if (dq > bmax) bmax = dq;
          if (dq < bmin) bmin = dq;
          cnt++;
        }
    int widen = 0;
    for (int a = 0; a < 3; a++)
      if (spread[a] < 0.5) {
        if (pass == 0) { w[a] = 2; widen = 1; }
        else return 1.0; /* still too narrow: zero gradient */
      }
    if (!widen) break;
  }
  if (cnt < 4) return 1.0;
  double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
               M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
  double tr = (M[0][0] + M[1][1] + M[2][2]) / 3.0;
  if (!(det > 1e-12 * tr * tr * tr)) return 1.0;
  /* Cramer's rule */
  for (int a = 0; a < 3; a++) {
    double A[3][3];
    memcpy(A, M, sizeof(A));
    for (int c = 0; c < 3; c++) A[c][a] = b[c];
    double da = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    sig[a] = da / det;
  }
  /* limiter at the centroids of the members of M_r */
  long mid[8];
  int moff[8][3];
  int nm = members(D, Gg, g, gi, gj, k, W->code[r], mid, moff);
  double phi = 1.0;
  for (int q = 0; q < nm; q++) {
    double xq[3], e[3], del = 0.0;
    for (int a = 0; a < 3; a++) xq[a] = moff[q][a] + Gg->cent[a * n + mid[q]];
    from_xhat(D, g, Gg, W, gi, gj, k, r, xq, e);
    for (int a = 0; a < 3; a++) del += sig[a] * e[a];
    double ph = 1.0;
    if (del > 0.0) ph = bmax / del;
    else if (del < 0.0) ph = bmin / del;
    if (ph > 1.0) ph = 1.0;
    if (ph < phi) phi = ph;
  }
  for (int a = 0; a < 3; a++) sig[a] *= phi;
  return phi;
}

/* Redistribution of one field of grid g (Eqs. qhat_omega, qrecon,
 * final_update_omega): Uhat -> Unew.  Inactive CVs are copied.  The final
 * update is written as U_i = P_i + (1/N_i) sum_{r in W-_i} kappa_r
 * (q_r(x_i) - P_i) with P_i = q_i(x_i), which is Eq. final_update_omega
 * because omega_i = 1 - (1/N_i) sum kappa_r (Eq. omega).  If sigma_out /
 * phi_out / qhat_out are not NULL they receive the limited gradient (3n), the
 * limiter factor (n, 1 where no gradient was fitted) and the neighbourhood
 * average Qhat of every CV (n; Uhat itself where the CV is not small). */
int orc_wsrd_apply(const OrcDomain *D, int g, const OrcGeom *Gg, const OrcWsrd *W, const double *Uh, double *Un,
                   double *sigma_out, double *phi_out, double *qhat_out) {
  long n = ncv(D, g);
  int nzg = nzg_of(D, g);
  long *piv = malloc(sizeof(long) * (size_t)n);
  double *Dv = malloc(sizeof(double) * (size_t)n);
  double *sg = calloc((size_t)n * 3, sizeof(double));
  QhatForm Q = {Uh, piv, Dv};
  /* neighbourhood averages (Eq. qhat_omega), pivoted deviation form */
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nzg; k++)
    for (int lj = 0; lj < D->WY; lj++)
      for (int li = 0; li < D->WX; li++) {
        long id = (long)li + (long)D->WX * ((long)lj + (long)D->WY * k);
        int gi = D->x0 + li, gj = D->y0 + lj;
        piv[id] = id;
        Dv[id] = 0.0;
        if (active(D, Gg, g, gi, gj, k) < 0 || W->code[id] == 0) continue;
        long mid[8];
        int moff[8][3];
        int nm = members(D, Gg, g, gi, gj, k, W->code[id], mid, moff);
        double wt[8];
        wt[0] = W->omega[id] * Gg->alpha[id] / W->vhat[id];
        for (int q = 1; q < nm; q++) wt[q] = W->kappa[id] * Gg->alpha[mid[q]] / W->nnb[mid[q]] / W->vhat[id];
        int p = -1, big = 0;
        for (int q = 0; q < nm; q++) {
          if (p < 0 && Gg->alpha[mid[q]] >= 0.5) p = q;
          if (Gg->alpha[mid[q]] > Gg->alpha[mid[big]]) big = q;
        }
        if (p < 0) p = big;
        double s = 0.0;
        for (int q = 0; q < nm; q++)
          if (q != p) s += wt[q] * (Uh[mid[q]] - Uh[mid[p]]);
        piv[id] = mid[p];
        Dv[id] = s;
      }
  /* gradients (small CVs whose neighbourhood holds at least two CVs) */
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nzg; k++)
    for (int lj = 0; lj < D->WY; lj++)
      for (int li = 0; li < D->WX; li++) {
        long id = (long)li + (long)D->WX * ((long)lj + (long)D->WY * k);
        int gi = D->x0 + li, gj = D->y0 + lj;
        double phi = 1.0;
        if (active(D, Gg, g, gi, gj, k) >= 0 && W->code[id] != 0) {
          long mid[8];
          int moff[8][3];
          int nm = members(D, Gg, g, gi, gj, k, W->code[id], mid, moff);
          if (nm >= 2) {
            double s3[3];
            phi = lsq_gradient(D, g, Gg, W, &Q, gi, gj, k, id, s3);
            for (int a = 0; a < 3; a++) sg[a * n + id] = s3[a];
          }
        }
        if (phi_out) phi_out[id] = phi;
      }
  /* final update (Eq. final_update_omega) */
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nzg; k++)
    for (int lj = 0; lj < D->WY; lj++)
      for (int li = 0; li < D->WX; li++) {
        long id = (long)li + (long)D->WX * ((long)lj + (long)D->WY * k);
        int gi = D->x0 + li, gj = D->y0 + lj;
        if (active(D, Gg, g, gi, gj, k) < 0) { Un[id] = Uh[id]; continue; }
        double xi[3] = {Gg->cent[id], Gg->cent[n + id], Gg->cent[2 * n + id]};
        /* own reconstruction at own centroid, as an offset from Uhat_i */
        double si = 0.0;
        if (W->code[id]) {
          double ei[3];
          from_xhat(D, g, Gg, W, gi, gj, k, id, xi, ei);
          for (int a = 0; a < 3; a++) si += sg[a * n + id] * ei[a];
        }
        double acc = 0.0;
        for (int dk = -1; dk <= 1; dk++)
          for (int dj = -1; dj <= 1; dj++)
            for (int di = -1; di <= 1; di++) {
              if (!di && !dj && !dk) continue;
              long r = active(D, Gg, g, gi + di, gj + dj, k + dk);
              if (r < 0 || W->code[r] == 0) continue;
              long mid[8];
              int moff[8][3];
              int nm = members(D, Gg, g, gi + di, gj + dj, k + dk, W->code[r], mid, moff);
              for (int qq = 1; qq < nm; qq++)
                if (moff[qq][0] == -di && moff[qq][1] == -dj && moff[qq][2] == -dk) {
                  /* q_r(x_i) - P_i, positions relative to r's centre */
                  double xir[3] = {-di + xi[0], -dj + xi[1], -dk + xi[2]}, er[3], sr = 0.0;
                  from_xhat(D, g, Gg, W, gi + di, gj + dj, k + dk, r, xir, er);
                  for (int a = 0; a < 3; a++) sr += sg[a * n + r] * er[a];
                  acc += W->kappa[r] * (qdiff(&Q, r, id) + sr - si);
                }
            }
        /* A small CV's result is anchored at its pivot, Uhat[piv] + D + s +
         * corrections: Uhat_i itself can be huge (a tiny cell after the flux
         * update) and must not be added and subtracted again. */
        if (W->code[id]) Un[id] = Uh[piv[id]] + ((Dv[id] + si) + acc / W->nnb[id]);
        else Un[id] = Uh[id] + acc / W->nnb[id];
      }
  if (sigma_out) memcpy(sigma_out, sg, sizeof(double) * (size_t)n * 3);
  if (qhat_out)
    for (long c = 0; c < n; c++) qhat_out[c] = Uh[piv[c]] + Dv[c];
  free(piv);
  free(Dv);
  free(sg);
  return 0;
}

/* ------------------------------------------------------------------------- */
/* 4. Sources of the compressible system (Sec. 2.1, Eq. mom-comp)            */
/* ------------------------------------------------------------------------- */
/* The momentum equation of the compressible system carries -grad p' and the
 * buoyancy B = -rho' g (g pointing down: a force -rho' |g| on rho*w), with
 * p' = p - p0(z), rho' = rho - rho0(z) and p from the equation of state
 * p = P00 (R rho theta / P00)^gamma; the reference state satisfies it,
 * p0 = P00 (R rho0 theta0 / P00)^gamma.  P00 = 1e5 Pa is the paper's; the gas
 * constant and specific heat of dry air and the gravitational acceleration
 * are not printed there: R = 287 J/(kg K), cp = 1004.5 J/(kg K),
 * gamma = cp / (cp - R), g = 9.81 m/s^2.
 *
 * On the staggered mesh the pressure and the density live at cell centres
 * and every momentum CV sits between two cells along its staggering axis d
 * (the cell below, e_d back, and the cell of the same index): the source of
 * the CV is the difference of p' across it over dx_d, and on w the mean of
 * rho' of the two cells.  The source enters dU of the CV as it stands (the
 * integral of a source over the CV over its volume).  A cell that is covered
 * (or outside the window) takes the value of the other cell: no pressure
 * force across a wall side, the buoyancy of the fluid cell. */
#define ORC_P00 1.0e5
#define ORC_RD 287.0
#define ORC_CP 1004.5

typedef struct {
  const double *rho0;   /* nz  reference density of every level              */
  const double *rt0;    /* nz  reference rho0*theta0 of every level          */
  double grav;          /* gravitational acceleration (buoyancy), m/s^2      */
  int pressure;         /* add -grad p'                                     */
  int buoyancy;         /* add -rho' g to rho*w                              */
} OrcSources;

/* p from the equation of state */
double orc_eos_pressure(double rt) {
  double gamma = ORC_CP / (ORC_CP - ORC_RD);
  return ORC_P00 * pow(ORC_RD * rt / ORC_P00, gamma);
}

/* p' = p(rt) - p(rt0) of a cell with rho*theta = rt on a level with
 * reference rt0.  Written as p(rt0) [(1 + x)^gamma - 1], x = (rt - rt0) / rt0,
 * the same quantity without subtracting two values near 1e5 Pa (which
 * would leave an error near 1e-11 Pa in p'); rt - rt0 is exact in FP64 for
 * rt within a factor two of rt0. */
static double pressure_perturbation(double rt, double rt0) {
  double gamma = ORC_CP / (ORC_CP - ORC_RD);
  return orc_eos_pressure(rt0) * expm1(gamma * log1p((rt - rt0) / rt0));
}

/* Adds the sources of state U to dU (rho*u, rho*v, rho*w; every prognostic
 * non-covered CV of the window). */
int orc_sources(const OrcDomain *D, const OrcGeom *G, const OrcState *U, const OrcSources *S, OrcState *dU) {
  const double inv[3] = {1.0 / D->dx, 1.0 / D->dy, 1.0 / D->dz};
  for (int g = GU; g <= GW; g++) {
    int d = g - 1, di = d == 0, dj = d == 1, dk = d == 2;
    int nzg = nzg_of(D, g);
    double *out = dU->f[g + 1];
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nzg; k++) {
      if (!prognostic(D, g, k)) continue;
      for (int wj = 0; wj < D->WY; wj++)
        for (int wi = 0; wi < D->WX; wi++) {
          int gi = D->x0 + wi, gj = D->y0 + wj;
          long id = avail(D, G, g, gi, gj, k);
          if (id < 0) continue;
          long a = avail(D, G, GC, gi - di, gj - dj, k - dk);   /* the cell below along d */
          long b = avail(D, G, GC, gi, gj, k);                    /* the cell of the same index */
          if (a < 0 && b < 0) continue;
          int ka = k - dk;
          double s = 0.0;
          if (S->pressure) {
            double pa = a >= 0 ? pressure_perturbation(U->f[1][a], S->rt0[ka]) : 0.0;
            double pb = b >= 0 ? pressure_perturbation(U->f[1][b], S->rt0[k]) : 0.0;
            if (a < 0) pa = pb;
            if (b < 0) pb = pa;
            s -= (pb - pa) * inv[d];
          }
          if (S->buoyancy && g == GW) {
            double ra = a >= 0 ? U->f[0][a] - S->rho0[ka] : 0.0;
            double rb = b >= 0 ? U->f[0][b] - S->rho0[k] : 0.0;
            if (a < 0) ra = rb;
            if (b < 0) rb = ra;
            s -= S->grav * 0.5 * (ra + rb);
          }
          out[id] += s;
        }
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* 5. The step (Algorithm 1)                                                   */
/* ------------------------------------------------------------------------- */
/* One stage: Uout = R[ Ubase + dt * (dU(Usrc) + S(Usrc)) ] on all four grids,
 * S the sources of section 4 (none when S is NULL).  scratch holds 5 arrays
 * of the field sizes. */
int orc_stage(const OrcDomain *D, const OrcGeom *G, const OrcWsrd *W, const OrcState *Usrc, const OrcState *Ubase,
              double dt, OrcState *Uout, OrcState *scratch, const OrcSources *S) {
  orc_flux_div(D, G, Usrc, scratch);
  if (S) orc_sources(D, G, Usrc, S, scratch);
  for (int f = 0; f < 5; f++) {
    int g = FIELD_GRID[f];
    long n = ncv(D, g);
    double *hat = scratch->f[f];
    for (long c = 0; c < n; c++) hat[c] = Ubase->f[f][c] + dt * hat[c];
    /* covered and non-prognostic CVs keep their value: dU is zero there */
    orc_wsrd_apply(D, g, &G[g], &W[g], hat, Uout->f[f], NULL, NULL, NULL);
  }
  return 0;
}

/* ------------------------------------------------------------------------- */
/* 6. Two-level static refinement (Sec. 4.3)                                  */
/* ------------------------------------------------------------------------- */
/* Refinement ratio 2 in every direction: the fine level has 2NX x 2NY x 2nz
 * cells over the same domain as the coarse one.  The coarse geometry is
 * built from the fine cells by merging, so that coarse volumes, face areas
 * and EB areas are sums of fine ones.  A coarse CV of any grid is a block of
 * 2x2x2 fine cells of the fine c grid: cells 2I, 2I+1 along x for the c grid,
 * 2I-1, 2I for the u grid (the right half of coarse cell I-1 and the left
 * half of cell I), likewise along y for v and along z for w; fine cells
 * below the bottom or above the top of the domain hold no fluid.
 *   volume fraction   the mean of the 8 fine ones;
 *   volume centroid   their volume-weighted mean position;
 *   face fraction     the mean of the 4 fine faces on the coarse low face,
 *                     its centroid their area-weighted mean position;
 *   EB area           the sum of the fine ones (a quarter of it in units of
 *                     the coarse dx dy), its centroid their area-weighted mean;
 *   EB normal         the direction of the area-weighted sum of the fine EB
 *                     normals, which (the boundary of a fluid region being
 *                     closed) is sum_d (open area of the high d-face - open
 *                     area of the low d-face) e_d over the coarse CV's faces;
 *   class             covered (all its fine cells inside the domain
 *                     covered), regular (all of them regular) or cut.
 * Positions are offsets from the CV (or face) centre in grid units of its
 * level: a fine cell's centre sits at -1/2 or +1/2 fine units from the
 * coarse CV centre along each axis, and a fine unit is half a coarse one. */

/* the fine c-grid cell (i, j, k) of the whole periodic fine domain; id < 0
 * outside the domain in z (no fluid) */
static long fine_id(const OrcDomain *Df, int i, int j, int k) {
  if (k < 0 || k >= Df->nz) return -1;
  return loc(Df, GC, imod(i, Df->NX), imod(j, Df->NY), k);
}

int orc_coarsen(const OrcDomain *Df, const OrcGeom *Gf, const OrcDomain *Dc, int g, OrcGeom *Gc) {
  if (Df->WX != Df->NX || Df->WY != Df->NY || Dc->WX != Dc->NX || Dc->WY != Dc->NY) return 1;
  if (Df->NX != 2 * Dc->NX || Df->NY != 2 * Dc->NY || Df->nz != 2 * Dc->nz) return 1;
  const OrcGeom *F = &Gf[GC];
  long nf = ncv(Df, GC), nc = ncv(Dc, g);
  int nzg = nzg_of(Dc, g);
  int sx = g == GU, sy = g == GV, sz = g == GW;
  double Af[3] = {Df->dy * Df->dz, Df->dx * Df->dz, Df->dx * Df->dy};
#pragma omp parallel for schedule(static)
  for (int K = 0; K < nzg; K++)
    for (int J = 0; J < Dc->NY; J++)
      for (int I = 0; I < Dc->NX; I++) {
        long id = loc(Dc, g, I, J, K);
        int f0[3] = {2 * I - sx, 2 * J - sy, 2 * K - sz};
        double vol = 0, m[3] = {0, 0, 0}, eba = 0, eb[3] = {0, 0, 0}, ebv[3] = {0, 0, 0};
        double fa[3] = {0, 0, 0}, f1[3] = {0, 0, 0}, f2[3] = {0, 0, 0}, fh[3] = {0, 0, 0};
        int nin = 0, ncov = 0, nreg = 0;
        for (int c = 0; c < 2; c++)
          for (int b = 0; b < 2; b++)
            for (int a = 0; a < 2; a++) {
              int q[3] = {a, b, c};
              double o[3] = {a - 0.5, b - 0.5, c - 0.5};
              long f = fine_id(Df, f0[0] + a, f0[1] + b, f0[2] + c);
              if (f < 0) continue;   /* outside the domain: no fluid, and no part of the class */
              nin++;
              if (F->flag[f] == ORC_COVERED) ncov++;
              if (F->flag[f] == ORC_REGULAR) nreg++;
              double al = F->alpha[f], ae = F->aeb[f];
              vol += al;
              eba += ae;
              for (int d = 0; d < 3; d++) {
                m[d] += al * (o[d] + F->cent[d * nf + f]);
                eb[d] += ae * (o[d] + F->ebc[d * nf + f]);
                ebv[d] += F->ebv[d * nf + f];
              }
              for (int d = 0; d < 3; d++) {
                if (q[d] != 0) continue;   /* the fine cells on the coarse low d-face */
                int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
                double be = F->beta[d * nf + f];
                fa[d] += be;
                f1[d] += be * (o[t1] + F->fcent[(2 * d) * nf + f]);
                f2[d] += be * (o[t2] + F->fcent[(2 * d + 1) * nf + f]);
              }
            }
        /* open areas of the coarse high faces: the low faces of the fine cells
         * two beyond the block's first; the lid above the top is open */
        for (int d = 0; d < 3; d++)
          for (int u = 0; u < 2; u++)
            for (int v = 0; v < 2; v++) {
              int ii = f0[0], jj = f0[1], kk = f0[2];
              int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
              int *pd = d == 0 ? &ii : d == 1 ? &jj : &kk;
              int *p1 = t1 == 0 ? &ii : &jj;
              int *p2 = t2 == 1 ? &jj : &kk;
              *pd += 2;
              *p1 += u;
              *p2 += v;
              long f = fine_id(Df, ii, jj, kk);
              if (f >= 0) fh[d] += F->beta[d * nf + f];
              else if (d == 2 && kk >= Df->nz) fh[d] += 1.0;
            }
        Gc->flag[id] = (uint8_t)(ncov == nin ? ORC_COVERED : nreg == nin ? ORC_REGULAR : ORC_CUT);
        Gc->alpha[id] = vol / 8.0;
        Gc->aeb[id] = eba / 4.0;
        double nv[3], nn = 0;
        for (int d = 0; d < 3; d++) {
          Gc->cent[d * nc + id] = vol > 0 ? 0.5 * m[d] / vol : 0.0;
          Gc->beta[d * nc + id] = fa[d] / 4.0;
          Gc->fcent[(2 * d) * nc + id] = fa[d] > 0 ? 0.5 * f1[d] / fa[d] : 0.0;
          Gc->fcent[(2 * d + 1) * nc + id] = fa[d] > 0 ? 0.5 * f2[d] / fa[d] : 0.0;
          Gc->ebc[d * nc + id] = eba > 0 ? 0.5 * eb[d] / eba : 0.0;
          Gc->ebv[d * nc + id] = ebv[d] / 4.0;
          nv[d] = (fh[d] - fa[d]) * Af[d];
          nn += nv[d] * nv[d];
        }
        nn = sqrt(nn);
        for (int d = 0; d < 3; d++) Gc->nrm[d * nc + id] = (eba > 0 && nn > 0) ? nv[d] / nn : 0.0;
      }
  return 0;
}

/* Restriction of a fine state to the coarse level (Sec. 4.3): a coarse
 * cell-centred value is the volume-weighted mean of its 8 fine cells (weights
 * the fine volume fractions), so that the coarse cell holds the fine cells'
 * total; a coarse face value is the area-weighted mean of the 4 fine values
 * on its face (weights the fine face fractions), so that the flux integral
 * over the coarse face is kept.  Only the coarse columns over the fine
 * columns [x_lo, x_hi) (global fine indices, both even, periodic) are
 * restricted; the fine domain may be a window holding them.  Coarse CVs whose
 * fine parts hold no fluid or no open area keep their values (Uc is read and
 * written). */
int orc_restrict(const OrcDomain *Df, const OrcGeom *Gf, const OrcState *Uf, const OrcDomain *Dc, OrcState *Uc,
                 int x_lo, int x_hi) {
  if (Df->NX != 2 * Dc->NX || Df->NY != 2 * Dc->NY || Df->nz != 2 * Dc->nz) return 1;
  if (x_lo % 2 || x_hi % 2 || x_hi <= x_lo || x_hi - x_lo > Df->NX) return 1;
  const OrcGeom *F = &Gf[GC];
  long nf = ncv(Df, GC);
  for (int fld = 0; fld < 5; fld++) {
    int g = FIELD_GRID[fld];
    int nzg = nzg_of(Dc, g);
    int d = g - 1;
#pragma omp parallel for schedule(static)
    for (int K = 0; K < nzg; K++)
      for (int J = 0; J < Dc->NY; J++)
        for (int Ix = x_lo / 2; Ix < x_hi / 2; Ix++) {
          int I = imod(Ix, Dc->NX);
          long id = loc(Dc, g, I, J, K);
          double w = 0, s = 0;
          if (g == GC) {
            for (int c = 0; c < 2; c++)
              for (int b = 0; b < 2; b++)
                for (int a = 0; a < 2; a++) {
                  long f = fine_id(Df, 2 * I + a, 2 * J + b, 2 * K + c);
                  w += F->alpha[f];
                  s += F->alpha[f] * Uf->f[fld][f];
                }
          } else {
            /* the 4 fine faces of grid g at fine index 2I (2J, 2K) along d */
            for (int v = 0; v < 2; v++)
              for (int u = 0; u < 2; u++) {
                int ii = 2 * I, jj = 2 * J, kk = 2 * K;
                if (d == 0) { jj += u; kk += v; }
                else if (d == 1) { ii += u; kk += v; }
                else { ii += u; jj += v; }
                long f = fine_id(Df, ii, jj, kk);          /* the fine cell whose low d-face it is */
                if (f < 0) continue;                        /* the top lid of w: a wall */
                long fu = loc(Df, g, imod(ii, Df->NX), imod(jj, Df->NY), kk);
                double be = F->beta[d * nf + f];
                w += be;
                s += be * Uf->f[fld][fu];
              }
          }
          if (w > 0) Uc->f[fld][id] = s / w;
        }
  }
  return 0;
}

/* Prolongation of a coarse state onto a fine window (the boundary values a
 * refined patch takes from the coarse level, Sec. 4.3): every fine CV of the
 * window outside the columns [x_lo, x_hi) (global fine indices, periodic)
 * takes the value of the coarse CV it lies in; a fine face of a face grid
 * that lies on a coarse face takes that face's value, one halfway between two
 * coarse faces (the odd fine index along the face's axis) their mean.  Covered
 * CVs included: the step passes them through. */
int orc_prolong(const OrcDomain *Dc, const OrcState *Uc, const OrcDomain *Df, OrcState *Uf, int x_lo, int x_hi) {
  if (Df->NX != 2 * Dc->NX || Df->NY != 2 * Dc->NY || Df->nz != 2 * Dc->nz) return 1;
  for (int fld = 0; fld < 5; fld++) {
    int g = FIELD_GRID[fld];
    int nzg = nzg_of(Df, g);
    int d = g - 1;
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nzg; k++)
      for (int wj = 0; wj < Df->WY; wj++)
        for (int wi = 0; wi < Df->WX; wi++) {
          int gi = Df->x0 + wi, gj = Df->y0 + wj;
          int rel = imod(gi - x_lo, Df->NX);
          if (rel < x_hi - x_lo) continue;   /* an owned column */
          int c[3] = {imod(gi, Df->NX) / 2, imod(gj, Df->NY) / 2, k / 2};
          int f[3] = {imod(gi, Df->NX), imod(gj, Df->NY), k};
          long id = loc(Df, g, gi, gj, k);
          double v;
          long a = loc(Dc, g, c[0], c[1], c[2]);
          if (g == GC || f[d] % 2 == 0) {
            v = Uc->f[fld][a];
          } else {
            int c2[3] = {c[0], c[1], c[2]};
            c2[d] += 1;
            if (d < 2) c2[d] = imod(c2[d], d == 0 ? Dc->NX : Dc->NY);
            v = 0.5 * (Uc->f[fld][a] + Uc->f[fld][loc(Dc, g, c2[0], c2[1], c2[2])]);
          }
          Uf->f[fld][id] = v;
        }
  }
  return 0;
}
