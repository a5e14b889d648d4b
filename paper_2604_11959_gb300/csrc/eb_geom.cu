// eb_geom.cu -- one-time cut-cell geometry of the four staggered grids
// (Sec. 3.2 of the paper), FP64.
//
// The EB is the nodal level set z - h: heights live on the lattice nodes and
// each lattice square is split along its (0,0)-(1,1) diagonal into two
// triangles on which h is linear.  The covered / regular / cut class of a CV
// comes from comparing the level set at the corners of its footprint with the
// CV's top and bottom levels (Sec. 3.2: the nodal level set classifies each
// cell).  Corner values are h_node / dz at lattice nodes and (Ha + Hb) * 0.5
// at edge and diagonal midpoints, so the classification is exact and
// reproducible.  Cut CVs then get their moments: fluid volume and centroid,
// open area and centroid of each face, and the EB area, area-weighted normal
// and centroid.  Face-grid CVs are the union of two half-cells of the
// cell-centred grid (Sec. 3.2, "two half-cells from neighboring cell-centered
// control volumes"): areas and volumes add, the normal and centroid are area
// weighted.  The z-face grid's two halves share one footprint, so a w CV is
// integrated as one box over [k - 1/2, k + 1/2], which is the same sum.
#include "eb_internal.cuh"
#include "eb_kernels.cuh"

#include <math.h>

namespace {

struct Poly {
  int n;
  double x[10], y[10], h[10];
};

// Half-lattice heights of lattice square (I, J) (periodic), in dz units.
__device__ void square_heights(const double *h, const Dims &D, int I, int J, double Hq[3][3]) {
  const int i0 = wrapi(I, D.nx), j0 = wrapi(J, D.ny);
  const long long W = D.nx + 1;
  const double a = h[(long long)j0 * W + i0] / D.dz;
  const double b = h[(long long)j0 * W + i0 + 1] / D.dz;
  const double c = h[(long long)(j0 + 1) * W + i0] / D.dz;
  const double e = h[(long long)(j0 + 1) * W + i0 + 1] / D.dz;
  Hq[0][0] = a;
  Hq[2][0] = b;
  Hq[0][2] = c;
  Hq[2][2] = e;
  Hq[1][0] = (a + b) * 0.5;
  Hq[1][2] = (c + e) * 0.5;
  Hq[0][1] = (a + c) * 0.5;
  Hq[2][1] = (b + e) * 0.5;
  Hq[1][1] = (a + e) * 0.5;
}

// Keep the part of a convex polygon with coordinate `axis` <= lim (le) or
// >= lim (!le).  Intersections land on half-lattice points here.
__device__ void cut_axis(const Poly &in, Poly &out, int axis, double lim, bool le) {
  out.n = 0;
  for (int e = 0; e < in.n; ++e) {
    const int f = (e + 1 == in.n) ? 0 : e + 1;
    const double ce = axis == 0 ? in.x[e] : in.y[e];
    const double cf = axis == 0 ? in.x[f] : in.y[f];
    const bool ie = le ? (ce <= lim) : (ce >= lim);
    const bool iff = le ? (cf <= lim) : (cf >= lim);
    if (ie) {
      out.x[out.n] = in.x[e];
      out.y[out.n] = in.y[e];
      out.h[out.n] = in.h[e];
      ++out.n;
    }
    if (ie != iff) {
      const double t = (lim - ce) / (cf - ce);
      out.x[out.n] = in.x[e] + t * (in.x[f] - in.x[e]);
      out.y[out.n] = in.y[e] + t * (in.y[f] - in.y[e]);
      out.h[out.n] = 0.0;
      ++out.n;
    }
  }
}

// Keep the part with height below lev (below) or at/above lev (!below).
__device__ void cut_level(const Poly &in, Poly &out, double lev, bool below) {
  out.n = 0;
  for (int e = 0; e < in.n; ++e) {
    const int f = (e + 1 == in.n) ? 0 : e + 1;
    const bool ie = below ? (in.h[e] < lev) : (in.h[e] >= lev);
    const bool iff = below ? (in.h[f] < lev) : (in.h[f] >= lev);
    if (ie) {
      out.x[out.n] = in.x[e];
      out.y[out.n] = in.y[e];
      out.h[out.n] = in.h[e];
      ++out.n;
    }
    if (ie != iff) {
      const double t = (lev - in.h[e]) / (in.h[f] - in.h[e]);
      out.x[out.n] = in.x[e] + t * (in.x[f] - in.x[e]);
      out.y[out.n] = in.y[e] + t * (in.y[f] - in.y[e]);
      out.h[out.n] = lev;
      ++out.n;
    }
  }
}

// Area and first moments of a simple polygon by Green's theorem, taken
// about its first vertex (a small polygon far from the origin keeps its
// centroid): m = {A, int x, int y}.
__device__ void green_moments(const Poly &p, double m[3]) {
  m[0] = m[1] = m[2] = 0.0;
  if (p.n < 3) return;
  const double ox = p.x[0], oy = p.y[0];
  for (int e = 1; e + 1 < p.n; ++e) {
    const double x0 = p.x[e] - ox, y0 = p.y[e] - oy, x1 = p.x[e + 1] - ox, y1 = p.y[e + 1] - oy;
    const double c = x0 * y1 - x1 * y0;
    m[0] += c;
    m[1] += (x0 + x1) * c;
    m[2] += (y0 + y1) * c;
  }
  m[0] *= 0.5;
  m[1] *= 1.0 / 6.0;
  m[2] *= 1.0 / 6.0;
  if (!(m[0] > 0.0)) {
    m[0] = m[1] = m[2] = 0.0;
    return;
  }
  m[1] += ox * m[0];
  m[2] += oy * m[0];
}

struct BoxMoments {
  double vol, mx, my, mz;
  double fa[6], f1[6], f2[6];  // xlo, xhi, ylo, yhi, zlo, zhi
  double eba, ebx, eby, ebz;
  double nv[3];
};

// One side of the footprint rectangle, as a vertical face: piecewise-linear
// height along s (half-lattice breakpoints), fluid height
// g(s) = clamp(Z1 - max(H, Z0), 0, Z1 - Z0).  Exact integrals of g, s*g and
// the z-moment over [b(s), Z1] with b = max(H, Z0).
__device__ void side_integrals(const double Hq[3][3], bool along_y, int c2, int s0, int s1, double Z0, double Z1,
                               double zb, double &A, double &S, double &Zm) {
  A = S = Zm = 0.0;
  for (int q = s0; q < s1; ++q) {
    const double sa = 0.5 * q, sb = 0.5 * (q + 1);
    const double Ha = along_y ? Hq[c2][q] : Hq[q][c2];
    const double Hb = along_y ? Hq[c2][q + 1] : Hq[q + 1][c2];
    double br[4];
    int nb = 0;
    br[nb++] = 0.0;
    double t0 = -1.0, t1 = -1.0;
    if ((Ha < Z0) != (Hb < Z0)) t0 = (Z0 - Ha) / (Hb - Ha);
    if ((Ha < Z1) != (Hb < Z1)) t1 = (Z1 - Ha) / (Hb - Ha);
    if (t0 >= 0.0 && t1 >= 0.0) {
      br[nb++] = fmin(t0, t1);
      br[nb++] = fmax(t0, t1);
    } else if (t0 >= 0.0) {
      br[nb++] = t0;
    } else if (t1 >= 0.0) {
      br[nb++] = t1;
    }
    br[nb++] = 1.0;
    for (int r = 0; r + 1 < nb; ++r) {
      const double ta = br[r], tb = br[r + 1];
      if (!(tb > ta)) continue;
      const double u0 = sa + ta * (sb - sa), u1 = sa + tb * (sb - sa);
      const double len = u1 - u0;
      const double Hm = Ha + 0.5 * (ta + tb) * (Hb - Ha);
      if (Hm >= Z1) continue;
      // base b(s) of the fluid column, linear on [u0, u1]
      double b0, b1;
      if (Hm < Z0) {
        b0 = b1 = Z0;
      } else {
        b0 = Ha + ta * (Hb - Ha);
        b1 = Ha + tb * (Hb - Ha);
      }
      const double g0 = Z1 - b0, g1 = Z1 - b1;
      A += 0.5 * len * (g0 + g1);
      S += len / 6.0 * (u0 * (2.0 * g0 + g1) + u1 * (g0 + 2.0 * g1));
      // z-moment of the column [b, Z1]: g (top - g/2), g linear on [u0, u1]
      const double top = Z1 - zb;
      Zm += top * 0.5 * len * (g0 + g1) - len / 6.0 * (g0 * g0 + g0 * g1 + g1 * g1);
    }
  }
}

// Moments of box [a0/2, a1/2] x [b0/2, b1/2] x [Z0, Z1] of square Hq.
// Coordinates: xi, eta local to the square, heights relative to zb.
__device__ void box_moments(const double Hq[3][3], int a0, int a1, int b0, int b1, double Z0, double Z1, double zb,
                            double sx, double sy, BoxMoments &M) {
  M.vol = M.mx = M.my = M.mz = 0.0;
  for (int f = 0; f < 6; ++f) M.fa[f] = M.f1[f] = M.f2[f] = 0.0;
  M.eba = M.ebx = M.eby = M.ebz = 0.0;
  M.nv[0] = M.nv[1] = M.nv[2] = 0.0;
  side_integrals(Hq, true, a0, b0, b1, Z0, Z1, zb, M.fa[0], M.f1[0], M.f2[0]);
  side_integrals(Hq, true, a1, b0, b1, Z0, Z1, zb, M.fa[1], M.f1[1], M.f2[1]);
  side_integrals(Hq, false, b0, a0, a1, Z0, Z1, zb, M.fa[2], M.f1[2], M.f2[2]);
  side_integrals(Hq, false, b1, a0, a1, Z0, Z1, zb, M.fa[3], M.f1[3], M.f2[3]);
  const double top = Z1 - zb;
  for (int t = 0; t < 2; ++t) {
    // triangle of the diagonal split and its plane H = p0 + px xi + py eta
    Poly tri;
    tri.n = 3;
    double px, py;
    if (t == 0) {
      tri.x[0] = 0; tri.y[0] = 0; tri.x[1] = 1; tri.y[1] = 0; tri.x[2] = 1; tri.y[2] = 1;
      px = Hq[2][0] - Hq[0][0];
      py = Hq[2][2] - Hq[2][0];
    } else {
      tri.x[0] = 0; tri.y[0] = 0; tri.x[1] = 1; tri.y[1] = 1; tri.x[2] = 0; tri.y[2] = 1;
      px = Hq[2][2] - Hq[0][2];
      py = Hq[0][2] - Hq[0][0];
    }
    Poly a, b;
    cut_axis(tri, a, 0, 0.5 * a0, false);
    cut_axis(a, b, 0, 0.5 * a1, true);
    cut_axis(b, a, 1, 0.5 * b0, false);
    cut_axis(a, b, 1, 0.5 * b1, true);
    if (b.n < 3) continue;
    for (int v = 0; v < b.n; ++v) b.h[v] = Hq[(int)(2.0 * b.x[v] + 0.25)][(int)(2.0 * b.y[v] + 0.25)];
    Poly rA, rB, rU, tmp;
    cut_level(b, rA, Z0, true);    // below the box: full height
    cut_level(b, tmp, Z0, false);
    cut_level(tmp, rB, Z1, true);  // EB inside the box
    cut_level(b, rU, Z1, true);    // open part of the top face
    double mA[3], mU[3];
    green_moments(rA, mA);
    green_moments(rU, mU);
    const double hgt = Z1 - Z0;
    M.vol += hgt * mA[0];
    M.mx += hgt * mA[1];
    M.my += hgt * mA[2];
    M.mz += 0.5 * (top * top - (Z0 - zb) * (Z0 - zb)) * mA[0];
    // region B: fluid height g = Z1 - H >= 0, linear; integrate over a fan of
    // triangles from the vertex values so that thin slivers (tiny g) keep
    // their relative accuracy: int f g = A/12 (sum f_i g_i + sum f_i sum g_i)
    double aB = 0.0, xB = 0.0, yB = 0.0, Ig = 0.0, Ixg = 0.0, Iyg = 0.0, Izm = 0.0;
    for (int q = 1; q + 1 < rB.n; ++q) {
      const int vi[3] = {0, q, q + 1};
      const double At = 0.5 * ((rB.x[q] - rB.x[0]) * (rB.y[q + 1] - rB.y[0]) -
                               (rB.x[q + 1] - rB.x[0]) * (rB.y[q] - rB.y[0]));
      if (!(At > 0.0)) continue;
      double g[3], xs[3], ys[3], zc[3];
      for (int v = 0; v < 3; ++v) {
        g[v] = Z1 - rB.h[vi[v]];
        xs[v] = rB.x[vi[v]];
        ys[v] = rB.y[vi[v]];
        zc[v] = top - 0.5 * g[v];   // mean height of the fluid column above the point, rel. zb
      }
      const double sg = g[0] + g[1] + g[2];
      aB += At;
      xB += At * (xs[0] + xs[1] + xs[2]) / 3.0;
      yB += At * (ys[0] + ys[1] + ys[2]) / 3.0;
      Ig += At * sg / 3.0;
      Ixg += At / 12.0 * (xs[0] * g[0] + xs[1] * g[1] + xs[2] * g[2] + (xs[0] + xs[1] + xs[2]) * sg);
      Iyg += At / 12.0 * (ys[0] * g[0] + ys[1] * g[1] + ys[2] * g[2] + (ys[0] + ys[1] + ys[2]) * sg);
      Izm += At / 12.0 * (zc[0] * g[0] + zc[1] * g[1] + zc[2] * g[2] + (zc[0] + zc[1] + zc[2]) * sg);
    }
    M.vol += Ig;
    M.mx += Ixg;
    M.my += Iyg;
    M.mz += Izm;
    M.fa[4] += mA[0]; M.f1[4] += mA[1]; M.f2[4] += mA[2];
    M.fa[5] += mU[0]; M.f1[5] += mU[1]; M.f2[5] += mU[2];
    if (aB > 0.0) {
      const double gx = sx * px, gy = sy * py;
      const double el = sqrt(1.0 + gx * gx + gy * gy);
      M.eba += el * aB;
      M.ebx += el * xB;
      M.eby += el * yB;
      M.ebz += el * (top * aB - Ig);   // EB height relative to zb: top - g
      M.nv[0] -= gx * aB;
      M.nv[1] -= gy * aB;
      M.nv[2] += aB;
    }
  }
}

// Covered / regular test of one box footprint against [Z0, Z1].
__device__ void box_minmax(const double Hq[3][3], int a0, int a1, int b0, int b1, double &mn, double &mx) {
  for (int a = a0; a <= a1; ++a)
    for (int b = b0; b <= b1; ++b) {
      mn = fmin(mn, Hq[a][b]);
      mx = fmax(mx, Hq[a][b]);
    }
}

// Footprint extremes of a CV column of grid g at column (i, j).
__device__ void column_minmax(const double *h, const Dims &D, int g, int i, int j, double &mn, double &mx) {
  double Hq[3][3];
  mn = 1e300;
  mx = -1e300;
  if (g == 1) {
    square_heights(h, D, i - 1, j, Hq);
    box_minmax(Hq, 1, 2, 0, 2, mn, mx);
    square_heights(h, D, i, j, Hq);
    box_minmax(Hq, 0, 1, 0, 2, mn, mx);
  } else if (g == 2) {
    square_heights(h, D, i, j - 1, Hq);
    box_minmax(Hq, 0, 2, 1, 2, mn, mx);
    square_heights(h, D, i, j, Hq);
    box_minmax(Hq, 0, 2, 0, 1, mn, mx);
  } else {
    square_heights(h, D, i, j, Hq);
    box_minmax(Hq, 0, 2, 0, 2, mn, mx);
  }
}

// Vertical extent of CV k of grid g, in dz units (w is cut by the walls).
__device__ inline void cv_levels(const Dims &D, int g, int k, double &Z0, double &Z1) {
  if (g == 3) {
    Z0 = fmax((double)k - 0.5, 0.0);
    Z1 = fmin((double)k + 0.5, (double)D.nz);
  } else {
    Z0 = (double)k;
    Z1 = (double)k + 1.0;
  }
}

struct CvSum {
  double vol, m[3], fa[3], f1[3], f2[3], eba, eb[3], nv[3];
};

__device__ void cv_add_box(CvSum &c, const BoxMoments &b, double ox, double oy, double oz, int fx, int fy, int fz) {
  c.vol += b.vol;
  c.m[0] += b.mx + ox * b.vol;
  c.m[1] += b.my + oy * b.vol;
  c.m[2] += b.mz + oz * b.vol;
  const int sel[3] = {fx, fy, fz};
  for (int d = 0; d < 3; ++d) {
    if (sel[d] < 0) continue;
    const int f = 2 * d + sel[d];
    const double o1 = d == 0 ? oy : ox;   // x faces: (y, z); y faces: (x, z); z faces: (x, y)
    const double o2 = d == 2 ? oy : oz;
    c.fa[d] += b.fa[f];
    c.f1[d] += b.f1[f] + o1 * b.fa[f];
    c.f2[d] += b.f2[f] + o2 * b.fa[f];
  }
  c.eba += b.eba;
  c.eb[0] += b.ebx + ox * b.eba;
  c.eb[1] += b.eby + oy * b.eba;
  c.eb[2] += b.ebz + oz * b.eba;
  for (int d = 0; d < 3; ++d) c.nv[d] += b.nv[d];
}

}  // namespace

// Geometry of CV (i, j, k) of grid g (cut or truncated wall CV): all moments
// in CV-centred cell units.  out[] = alpha, cent[3], beta[3], fcent[6],
// nrm[3], aeb, ebc[3] (20 values).
__device__ void cv_geometry(const double *h, const Dims &D, int g, int i, int j, int k, double out[20]) {
  CvSum c;
  c.vol = c.eba = 0.0;
  for (int d = 0; d < 3; ++d) c.m[d] = c.fa[d] = c.f1[d] = c.f2[d] = c.eb[d] = c.nv[d] = 0.0;
  const double sx = D.dz / D.dx, sy = D.dz / D.dy;
  double Hq[3][3];
  BoxMoments b;
  const double zb = (double)k;
  if (g == 0) {
    square_heights(h, D, i, j, Hq);
    box_moments(Hq, 0, 2, 0, 2, k, k + 1.0, zb, sx, sy, b);
    cv_add_box(c, b, -0.5, -0.5, -0.5, 0, 0, 0);
  } else if (g == 1) {
    square_heights(h, D, i - 1, j, Hq);
    box_moments(Hq, 1, 2, 0, 2, k, k + 1.0, zb, sx, sy, b);
    cv_add_box(c, b, -1.0, -0.5, -0.5, 0, 0, 0);
    square_heights(h, D, i, j, Hq);
    box_moments(Hq, 0, 1, 0, 2, k, k + 1.0, zb, sx, sy, b);
    cv_add_box(c, b, 0.0, -0.5, -0.5, -1, 0, 0);
  } else if (g == 2) {
    square_heights(h, D, i, j - 1, Hq);
    box_moments(Hq, 0, 2, 1, 2, k, k + 1.0, zb, sx, sy, b);
    cv_add_box(c, b, -0.5, -1.0, -0.5, 0, 0, 0);
    square_heights(h, D, i, j, Hq);
    box_moments(Hq, 0, 2, 0, 1, k, k + 1.0, zb, sx, sy, b);
    cv_add_box(c, b, -0.5, 0.0, -0.5, 0, -1, 0);
  } else {
    double Z0, Z1;
    cv_levels(D, 3, k, Z0, Z1);
    square_heights(h, D, i, j, Hq);
    box_moments(Hq, 0, 2, 0, 2, Z0, Z1, zb, sx, sy, b);
    // the low z face of the wall CV k = 0 lies on the domain wall: not a face
    cv_add_box(c, b, -0.5, -0.5, 0.0, 0, 0, k == 0 ? -1 : 0);
  }
  out[0] = c.vol;
  for (int d = 0; d < 3; ++d) {
    out[1 + d] = c.vol > 0.0 ? c.m[d] / c.vol : 0.0;
    out[4 + d] = c.fa[d];
    out[7 + 2 * d] = c.fa[d] > 0.0 ? c.f1[d] / c.fa[d] : 0.0;
    out[8 + 2 * d] = c.fa[d] > 0.0 ? c.f2[d] / c.fa[d] : 0.0;
    out[17 + d] = c.eba > 0.0 ? c.eb[d] / c.eba : 0.0;
  }
  const double nn = sqrt(c.nv[0] * c.nv[0] + c.nv[1] * c.nv[1] + c.nv[2] * c.nv[2]);
  for (int d = 0; d < 3; ++d) out[13 + d] = nn > 0.0 ? c.nv[d] / nn : 0.0;
  out[16] = c.eba;
}

// Class of CV k of grid g at a column with footprint extremes [mn, mx].
__device__ int cv_class(const Dims &D, int g, int k, double mn, double mx) {
  double Z0, Z1;
  cv_levels(D, g, k, Z0, Z1);
  if (mn >= Z1) return EBK_COVERED;
  if (mx < Z0) return EBK_REGULAR;
  return EBK_CUT;
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// Per column: first non-covered level and first level of the regular top.
__global__ void k_band_bounds(const double *h, Dims D, int g, int *kcov, int *kreg) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= D.nx * D.ny) return;
  const int i = col % D.nx, j = col / D.nx;
  double mn, mx;
  column_minmax(h, D, g, i, j, mn, mx);
  const int nzg = nzg_of(D, g);
  int kc = 0;
  while (kc < nzg && cv_class(D, g, kc, mn, mx) == EBK_COVERED) ++kc;
  int kr = nzg;
  while (kr > kc && cv_class(D, g, kr - 1, mn, mx) == EBK_REGULAR) --kr;
  kcov[col] = kc;
  kreg[col] = kr;
}

// Band top: one level above the highest non-regular CV of the 3x3 columns
// around, so that every member of a merging neighbourhood has a record.
__global__ void k_band_top(Dims D, int nzg, const int *kcov, const int *kreg, int *kxt, long long *count) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= D.nx * D.ny) return;
  const int i = col % D.nx, j = col / D.nx;
  int top = 0;
  for (int dj = -1; dj <= 1; ++dj)
    for (int di = -1; di <= 1; ++di) top = max(top, kreg[wrapi(i + di, D.nx) + D.nx * wrapi(j + dj, D.ny)]);
  top = min(nzg, top + 1);
  top = max(top, kcov[col]);
  kxt[col] = top;
  count[col] = top - kcov[col];
}

// First level of grid g's column from which every CV holds fluid (alpha > 0,
// the availability test of the flux stencils): the covered levels and any
// record without fluid lie below it.
__global__ void k_fluid_level(Dims D, GridDev G, int *kflu) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= D.nx * D.ny) return;
  const int kc = G.kcov[col];
  int kf = kc;
  for (int k = kc; k < G.kxt[col]; ++k)
    if (!(G.alpha[G.roff[col] + (k - kc)] > 0.0)) kf = k + 1;
  kflu[col] = kf;
}

// First level of the geometry-free path, shared by all grids.  From it up,
// the CVs of all four grids in the column are regular, and every CV that
// their flux stencils read (Sec. 4.1: up to three columns across, through the
// staggered averages, and three levels down, through the w-grid's advected
// values) holds fluid, so that every availability test passes and the plain
// stencil is the scheme's flux.  At least level 3, so that no stencil reaches
// the bottom wall.
__global__ void k_fast_level(Dims D, const int *kreg0, const int *kreg1, const int *kreg2, const int *kreg3,
                             const int *kflu0, const int *kflu1, const int *kflu2, const int *kflu3,
                             int *kfast) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= D.nx * D.ny) return;
  const int i = col % D.nx, j = col / D.nx;
  const int reg = max(max(kreg0[col], kreg1[col]), max(kreg2[col], kreg3[col]));
  int flu = 0;
  for (int dj = -3; dj <= 3; ++dj)
    for (int di = -3; di <= 3; ++di) {
      const int c = wrapi(i + di, D.nx) + D.nx * wrapi(j + dj, D.ny);
      flu = max(flu, max(max(kflu0[c], kflu1[c]), max(kflu2[c], kflu3[c])));
    }
  kfast[col] = min(D.nz, max(3, max(reg, flu + 3)));
}

// Geometry records of the band of every column.
__global__ void k_band_geometry(const double *h, Dims D, int g, GridDev G) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= D.nx * D.ny) return;
  const int i = col % D.nx, j = col / D.nx;
  double mn, mx;
  column_minmax(h, D, g, i, j, mn, mx);
  const long long n = G.nrec;
  for (int k = G.kcov[col]; k < G.kxt[col]; ++k) {
    const long long r = G.roff[col] + (k - G.kcov[col]);
    const int cls = cv_class(D, g, k, mn, mx);
    double v[20];
    if (cls == EBK_REGULAR && !(g == 3 && (k == 0 || k == D.nz))) {
      for (int q = 0; q < 20; ++q) v[q] = 0.0;
      v[0] = 1.0;
      v[4] = v[5] = v[6] = 1.0;
    } else {
      cv_geometry(h, D, g, i, j, k, v);
    }
    G.flag[r] = (uint8_t)cls;
    G.alpha[r] = v[0];
    for (int d = 0; d < 3; ++d) {
      G.cent[d * n + r] = v[1 + d];
      G.beta[d * n + r] = v[4 + d];
      G.nrm[d * n + r] = v[13 + d];
      G.ebc[d * n + r] = v[17 + d];
    }
    for (int q = 0; q < 6; ++q) G.fcent[q * n + r] = v[7 + q];
    G.aeb[r] = v[16];
    G.alpha_f[r] = (float)v[0];
    for (int d = 0; d < 3; ++d) G.beta_f[d * n + r] = (float)v[4 + d];
    for (int q = 0; q < 6; ++q) G.fcent_f[q * n + r] = (float)v[7 + q];
  }
}

// Dense availability / record byte of every CV of grid g.
__global__ void k_dense_flags(Dims D, int g, GridDev G) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= D.nx * D.ny) return;
  const int kc = G.kcov[col], kx = G.kxt[col];
  for (int k = 0; k < G.nzg; ++k) {
    uint8_t f = 0;
    if (k >= kx) {
      f = 1 | (7 << 2);   // regular: fluid, all three low faces open
    } else if (k >= kc) {
      const long long r = G.roff[col] + (k - kc);
      f = (uint8_t)(2 | (G.alpha[r] > 0.0 ? 1 : 0));
      for (int d = 0; d < 3; ++d)
        if (G.beta[d * G.nrec + r] > 0.0) f |= (uint8_t)(1 << (2 + d));
    }
    G.dflag[(long long)col + D.nxy * k] = f;
  }
}

// Band-list marks, plane-major: 1 for the CVs the near-EB kernel updates.
__global__ void k_band_marks(Dims D, int g, const int *kcov, const int *kfast, int kmax, long long *mark) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long ncol = D.nxy;
  if (t >= ncol * kmax) return;
  const int col = (int)(t % ncol), k = (int)(t / ncol);
  const int top = min(kfast[col], nzg_of(D, g));
  bool m = k >= kcov[col] && k < top;
  if (g == 3 && (k == 0 || k == D.nz)) m = false;
  mark[t] = m ? 1 : 0;
}

__global__ void k_band_fill(Dims D, int g, const int *kcov, const int *kfast, int kmax, const long long *pos,
                            unsigned *list) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long ncol = D.nxy;
  if (t >= ncol * kmax) return;
  const int col = (int)(t % ncol), k = (int)(t / ncol);
  const int top = min(kfast[col], nzg_of(D, g));
  bool m = k >= kcov[col] && k < top;
  if (g == 3 && (k == 0 || k == D.nz)) m = false;
  if (m) list[pos[t]] = (unsigned)(col + ncol * k);
}

// Faces whose provisional flux the near-EB path reads: the open low and
// high faces of every listed CV and the neighbour faces their centroid
// interpolation may use.  Several threads may mark the same face (all write 1).
__device__ inline bool face_open_dense(const Dims &D, const GridDev &G, int g, int d, int i, int j, int k) {
  if (k < 0 || k >= G.nzg) return false;
  if (g == 3 && d != 2 && (k < 1 || k > D.nz - 1)) return false;
  if (g != 3 && d == 2 && k == 0) return false;
  const long long c = (long long)wrapi(i, D.nx) + (long long)D.nx * wrapi(j, D.ny) + D.nxy * k;
  return (G.dflag[c] >> (2 + d)) & 1;
}

__global__ void k_face_marks(Dims D, int g, GridDev G, uint8_t *m0, uint8_t *m1, uint8_t *m2) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= G.nband) return;
  const long long p = G.blist[t];
  const int i = (int)(p % D.nx), j = (int)((p / D.nx) % D.ny), k = (int)(p / D.nxy);
  uint8_t *mk[3] = {m0, m1, m2};
  for (int d = 0; d < 3; ++d) {
    for (int h = 0; h < 2; ++h) {
      const int qi = i + (h && d == 0), qj = j + (h && d == 1), qk = k + (h && d == 2);
      if (h && d == 2 && g != 3 && qk >= D.nz) continue;   // top wall
      if (!face_open_dense(D, G, g, d, qi, qj, qk)) continue;
      const long long q = (long long)wrapi(qi, D.nx) + (long long)D.nx * wrapi(qj, D.ny) + D.nxy * qk;
      mk[d][q] = 1;
      if (!((G.dflag[q] >> 1) & 1)) continue;
      const int col = wrapi(qi, D.nx) + D.nx * wrapi(qj, D.ny);
      const long long r = G.roff[col] + (qk - G.kcov[col]);
      const double ga = G.fcent[(2 * d) * G.nrec + r], gb = G.fcent[(2 * d + 1) * G.nrec + r];
      const int ta = d == 0 ? 1 : 0, tb = d == 2 ? 1 : 2;
      int ea[3] = {0, 0, 0}, eb[3] = {0, 0, 0};
      ea[ta] = ga >= 0.0 ? 1 : -1;
      eb[tb] = gb >= 0.0 ? 1 : -1;
      for (int n = 1; n < 4; ++n) {
        if ((n & 1) && ga == 0.0) continue;
        if ((n & 2) && gb == 0.0) continue;
        const int ni = qi + ((n & 1) ? ea[0] : 0) + ((n & 2) ? eb[0] : 0);
        const int nj = qj + ((n & 1) ? ea[1] : 0) + ((n & 2) ? eb[1] : 0);
        const int nk = qk + ((n & 1) ? ea[2] : 0) + ((n & 2) ? eb[2] : 0);
        if (!face_open_dense(D, G, g, d, ni, nj, nk)) continue;
        mk[d][(long long)wrapi(ni, D.nx) + (long long)D.nx * wrapi(nj, D.ny) + D.nxy * nk] = 1;
      }
    }
  }
}

__global__ void k_marks_to_counts(const uint8_t *m, long long n, long long *cnt) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < n) cnt[t] = m[t];
}

__global__ void k_marks_fill(const uint8_t *m, long long n, const long long *pos, unsigned *list) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t < n && m[t]) list[pos[t]] = (unsigned)t;
}

// Dense export of one geometry field of one grid.
__global__ void k_export_geometry(const double *h, Dims D, int g, GridDev G, int field, double *dst) {
  const long long nzg = nzg_of(D, g);
  const long long total = D.nxy * nzg;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < total;
       c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(c % D.nx), j = (int)((c / D.nx) % D.ny), k = (int)(c / D.nxy);
    const CvInfo ci = cv_info(G, D, i, j, k);
    double v = 0.0;
    const bool wall = g == 3 && k == D.nz;
    if (field == EB_X_FLAG) {
      if (wall) {
        double mn, mx;
        column_minmax(h, D, g, i, j, mn, mx);
        v = cv_class(D, g, k, mn, mx);
      } else {
        v = ci.flag;
      }
    } else if (field <= EB_X_EBC_Z) {
      double vals[20];
      if (wall) {
        cv_geometry(h, D, g, i, j, k, vals);
      } else if (ci.rec >= 0) {
        const long long n = G.nrec, r = ci.rec;
        vals[0] = G.alpha[r];
        for (int d = 0; d < 3; ++d) {
          vals[1 + d] = G.cent[d * n + r];
          vals[4 + d] = G.beta[d * n + r];
          vals[13 + d] = G.nrm[d * n + r];
          vals[17 + d] = G.ebc[d * n + r];
        }
        for (int q = 0; q < 6; ++q) vals[7 + q] = G.fcent[q * n + r];
        vals[16] = G.aeb[r];
      } else {
        const bool reg = ci.flag == EBK_REGULAR;
        for (int q = 0; q < 20; ++q) vals[q] = 0.0;
        if (reg) vals[0] = vals[4] = vals[5] = vals[6] = 1.0;
      }
      // field order of the export enum: alpha, cent[3], beta[3], fcent[6], aeb, nrm[3], ebc[3]
      const int map[20] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 16, 13, 14, 15, 17, 18, 19};
      v = vals[map[field]];
    } else {
      // redistribution fields
      const long long n = G.nrec, r = ci.rec;
      const bool act = ci.flag != EBK_COVERED && !(g == 3 && (k == 0 || k == D.nz));
      if (field == EB_X_CODE) v = r >= 0 ? G.code[r] : 0.0;
      else if (field == EB_X_NNB) v = !act ? 0.0 : r >= 0 ? G.nnb[r] : 1.0;
      else if (field == EB_X_KAPPA) v = r >= 0 ? G.kappa[r] : 0.0;
      else if (field == EB_X_OMEGA) v = !act ? 0.0 : r >= 0 ? G.omega[r] : 1.0;
      else if (field == EB_X_VHAT) v = !act ? 0.0 : r >= 0 ? G.vhat[r] : 1.0;
      else if (field >= EB_X_XHAT_X && field <= EB_X_XHAT_Z) v = r >= 0 ? G.xhat[(field - EB_X_XHAT_X) * n + r] : 0.0;
    }
    dst[c] = v;
  }
}

// ---------------------------------------------------------------------------
// host wrappers
// ---------------------------------------------------------------------------
static inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

void launch_band_bounds(const double *h, const Dims &D, int g, int *kcov, int *kreg, cudaStream_t s) {
  k_band_bounds<<<nblk((long long)D.nx * D.ny, 128), 128, 0, s>>>(h, D, g, kcov, kreg);
}

void launch_band_top(const Dims &D, int nzg, const int *kcov, const int *kreg, int *kxt, long long *count,
                     cudaStream_t s) {
  k_band_top<<<nblk((long long)D.nx * D.ny, 256), 256, 0, s>>>(D, nzg, kcov, kreg, kxt, count);
}

void launch_fluid_level(const Dims &D, const GridDev &G, int *kflu, cudaStream_t s) {
  k_fluid_level<<<nblk((long long)D.nx * D.ny, 256), 256, 0, s>>>(D, G, kflu);
}

void launch_fast_level(const Dims &D, const int *const kreg[4], const int *const kflu[4], int *kfast,
                       cudaStream_t s) {
  k_fast_level<<<nblk((long long)D.nx * D.ny, 256), 256, 0, s>>>(D, kreg[0], kreg[1], kreg[2], kreg[3], kflu[0],
                                                                   kflu[1], kflu[2], kflu[3], kfast);
}

void launch_band_geometry(const double *h, const Dims &D, int g, const GridDev &G, cudaStream_t s) {
  k_band_geometry<<<nblk((long long)D.nx * D.ny, 64), 64, 0, s>>>(h, D, g, G);
}

void launch_export_geometry(const double *h, const Dims &D, int g, const GridDev &G, int field, double *dst,
                            cudaStream_t s) {
  const long long total = D.nxy * nzg_of(D, g);
  int blocks = nblk(total, 256);
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_export_geometry<<<blocks, 256, 0, s>>>(h, D, g, G, field, dst);
}

void launch_dense_flags(const Dims &D, int g, const GridDev &G, cudaStream_t s) {
  k_dense_flags<<<nblk((long long)D.nx * D.ny, 128), 128, 0, s>>>(D, g, G);
}

void launch_band_marks(const Dims &D, int g, const int *kcov, const int *kfast, int kmax, long long *mark,
                       cudaStream_t s) {
  const long long n = D.nxy * kmax;
  k_band_marks<<<nblk(n, 256), 256, 0, s>>>(D, g, kcov, kfast, kmax, mark);
}

void launch_band_fill(const Dims &D, int g, const int *kcov, const int *kfast, int kmax, const long long *pos,
                      unsigned *list, cudaStream_t s) {
  const long long n = D.nxy * kmax;
  k_band_fill<<<nblk(n, 256), 256, 0, s>>>(D, g, kcov, kfast, kmax, pos, list);
}

void launch_face_marks(const Dims &D, int g, const GridDev &G, uint8_t *m0, uint8_t *m1, uint8_t *m2, cudaStream_t s) {
  if (G.nband) k_face_marks<<<nblk(G.nband, 128), 128, 0, s>>>(D, g, G, m0, m1, m2);
}

void launch_marks_to_counts(const uint8_t *m, long long n, long long *cnt, cudaStream_t s) {
  k_marks_to_counts<<<nblk(n, 256), 256, 0, s>>>(m, n, cnt);
}

void launch_marks_fill(const uint8_t *m, long long n, const long long *pos, unsigned *list, cudaStream_t s) {
  k_marks_fill<<<nblk(n, 256), 256, 0, s>>>(m, n, pos, list);
}
