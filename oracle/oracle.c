/*
 * FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Plain restatement of arXiv 1912.11908 for a 2-D uniform Cartesian block.
 * The paper's solver is a curvilinear multi-block code; this oracle keeps the
 * parts of the method that act on one uniform block:
 *   Sec. 2      WENO5 reconstruction, low-diffusion flux splitting, central
 *               viscous flux
 *   Sec. 3.2    ray-casting node classification, IB and ghost tagging
 *   Sec. 4.1    closest surface feature (point-segment distance, Eq. 1 in 2-D)
 *   Sec. 4.2    pseudo-normals (Eq. 2 / Eq. 3 restricted to a polyline)
 *   Sec. 4.3    reconstruction along the local normal
 *   Sec. 4.4    boundary conditions (Eq. 4, 5, 6, 8)
 *   Sec. 4.6    inverse-distance-weighted interpolation
 *   Sec. 5      three ghost layers filled through image points
 *   Sec. 6      surface force integral (Eq. 9)
 * Readings where the paper is silent are written next to each routine.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NG 3 /* halo / ghost layers needed by the five-point WENO stencil (Sec. 5) */

struct orc_case {
  orc_params p;
  double *vref;            /* reference vertices, 2*nv */
  double *vx, *vy;         /* vertices at the current pose */
  double *snx, *sny;       /* outward segment normals */
  double *vnx, *vny;       /* vertex pseudo-normals */
  double *vk;              /* signed curvature at each vertex (convex > 0) */
  double dx, dy, h, dmin;
  double R, cp, mu, kappa, pinf;
  double Uinf[4];
  int W, H;
  double *A[4], *B[4], *C[4];
  double *q[4];            /* reconstructed primitives rho, u, v, p over the full array */
  double *T;               /* temperature over the full array */
  double *fx[4], *fy[4];   /* face fluxes */
  int precond;             /* low-Mach scaling of the dissipation (dual time only) */
  double *Wn[4], *Wm[4];   /* dual time: conserved state at time levels n and n-1 */
  long nphys;              /* dual time: physical steps taken (BDF1 on the first) */
  uint8_t *tag;
  int nlist[4];
  orc_stencil *list[4];
  double t, last_dt;
  int classified;
  int nerr;
  double pos[2];           /* body displacement at the classification time */
  /* body free to translate under the fluid force (Eq. 10): displacement, velocity and acceleration at bt, */
  /* the start of the current step, and the force that set the acceleration                                */
  double bX[2], bV[2], bA[2], bF[2], bt;
  double *snx0, *sny0, *vnx0, *vny0;  /* PITCH: normals of the reference pose */
};

static inline int fidx(const orc_case *c, int i, int j) { return (j + NG) * c->W + (i + NG); }

/* nodes the flux update advances: fluid nodes, and IB nodes when they are not rebuilt */
static inline int advanced(const orc_case *c, uint8_t tag) {
  return tag == ORC_FLUID || (tag == ORC_IB && c->p.ib_mode == ORC_IB_ADVANCE);
}

/* ------------------------------------------------------------------------- */
/* body motion: prescribed translation (Sec. 8.2.2 oscillating cylinder;     */
/* constant-velocity translation for the Galilean check of Sec. 8.2.3), or   */
/* translation under the fluid force (Sec. 6, Eq. 10): within a step the     */
/* body moves with the constant acceleration set at the step's start         */
/* ------------------------------------------------------------------------- */
static void motion_at(const orc_case *c, double t, double X[2], double V[2], double Acc[2]) {
  const orc_params *p = &c->p;
  X[0] = X[1] = V[0] = V[1] = Acc[0] = Acc[1] = 0.0;
  if (p->motion == ORC_MOTION_COUPLED) {
    double tau = t - c->bt;
    for (int k = 0; k < 2; k++) {
      Acc[k] = c->bA[k];
      V[k] = c->bV[k] + tau * c->bA[k];
      X[k] = c->bX[k] + tau * c->bV[k] + 0.5 * tau * tau * c->bA[k];
    }
  } else if (p->motion == ORC_MOTION_SIN) {
    double w = 2.0 * M_PI * p->freq;
    double s = sin(w * t), co = cos(w * t);
    for (int k = 0; k < 2; k++) {
      X[k] = p->amp[k] * s;
      V[k] = p->amp[k] * w * co;
      Acc[k] = -p->amp[k] * w * w * s;
    }
  } else if (p->motion == ORC_MOTION_CONST) {
    for (int k = 0; k < 2; k++) {
      X[k] = p->vel[k] * t;
      V[k] = p->vel[k];
    }
  }
}

/* pitching rotation (Sec. 7.2): body angle theta = -alpha(t) (counter-clockwise positive), its rate and     */
/* its acceleration                                                                                         */
static void pitch_at(const orc_case *c, double t, double *th, double *om, double *al) {
  const orc_params *p = &c->p;
  double w = 2.0 * M_PI * p->freq;
  *th = -(p->pitch_mean - p->pitch_amp * cos(w * t));
  *om = -p->pitch_amp * w * sin(w * t);
  *al = -p->pitch_amp * w * w * cos(w * t);
}

/* wall velocity and acceleration at the surface point (px, py): the translation's, plus for a pitching body  */
/* the rigid rotation about the pivot, V = om x r and A = al x r - om^2 r                                      */
static void wall_kin(const orc_case *c, double t, double px, double py, const double V0[2], const double A0[2],
                     double V[2], double A[2]) {
  if (c->p.motion != ORC_MOTION_PITCH) {
    V[0] = V0[0]; V[1] = V0[1];
    A[0] = A0[0]; A[1] = A0[1];
    return;
  }
  double th, om, al;
  pitch_at(c, t, &th, &om, &al);
  double rx = px - c->p.pivot[0], ry = py - c->p.pivot[1];
  V[0] = V0[0] - om * ry;
  V[1] = V0[1] + om * rx;
  A[0] = A0[0] - al * ry - om * om * rx;
  A[1] = A0[1] + al * rx - om * om * ry;
}

/* ------------------------------------------------------------------------- */
/* Sec. 3.2: ray-casting classification.  A ray is cast from the node along  */
/* +x; an odd number of crossings marks the node solid.  Reading of the      */
/* crossing test for a polyline: segment A->B is crossed iff                 */
/* (A.y > P.y) != (B.y > P.y) (half-open in y so a vertex on the ray counts  */
/* once) and the crossing abscissa lies strictly right of P.  Nodes outside  */
/* the axis-aligned bounding box are fluid without a test (Sec. 3.2).        */
/* ------------------------------------------------------------------------- */
static int point_in_body(int nv, const double *vx, const double *vy, const double bb[4], double px,
                         double py) {
  if (px < bb[0] || px > bb[1] || py < bb[2] || py > bb[3]) return 0;
  int odd = 0;
  for (int k = 0; k < nv; k++) {
    int k1 = (k + 1 == nv) ? 0 : k + 1;
    double ax = vx[k], ay = vy[k], bx = vx[k1], by = vy[k1];
    if ((ay > py) != (by > py)) {
      double t1 = py - ay;
      double t2 = bx - ax;
      double t3 = by - ay;
      double xint = ax + (t1 * t2) / t3;
      if (xint > px) odd ^= 1;
    }
  }
  return odd;
}

static void bbox(int nv, const double *vx, const double *vy, double bb[4]) {
  bb[0] = bb[1] = vx[0];
  bb[2] = bb[3] = vy[0];
  for (int k = 1; k < nv; k++) {
    if (vx[k] < bb[0]) bb[0] = vx[k];
    if (vx[k] > bb[1]) bb[1] = vx[k];
    if (vy[k] < bb[2]) bb[2] = vy[k];
    if (vy[k] > bb[3]) bb[3] = vy[k];
  }
}

void orc_classify_points(int nv, const double *verts, int np, const double *pts, uint8_t *solid) {
  double *vx = malloc(sizeof(double) * nv), *vy = malloc(sizeof(double) * nv);
  for (int k = 0; k < nv; k++) {
    vx[k] = verts[2 * k];
    vy[k] = verts[2 * k + 1];
  }
  double bb[4];
  bbox(nv, vx, vy, bb);
  for (int n = 0; n < np; n++) solid[n] = (uint8_t)point_in_body(nv, vx, vy, bb, pts[2 * n], pts[2 * n + 1]);
  free(vx);
  free(vy);
}

/* ------------------------------------------------------------------------- */
/* Sec. 3.2, 3-D: ray casting against a closed triangulated surface with the  */
/* Moller-Trumbore ray/triangle test: the ray hits a triangle when the       */
/* barycentric coordinates of its crossing with the triangle's plane are    */
/* all non-negative and the crossing lies ahead of the node.  For a ray      */
/* along a coordinate axis the unnormalised barycentric coordinates are the */
/* three edge functions of the triangle projected along the ray,            */
/*   E_ab(P) = (b_u - a_u)(P_v - a_v) - (b_v - a_v)(P_u - a_u),             */
/* each divided by the projected area; (u, v) the other two coordinates in  */
/* cyclic order.  Reading (the paper is silent on rays through an edge or a */
/* vertex, where inclusive bounds count a crossing twice and exclusive ones */
/* not at all): every edge function is evaluated with the edge's endpoints  */
/* in increasing vertex index, so the two triangles sharing an edge see     */
/* exactly opposite values, and a zero takes the sign of a symbolic shift   */
/* of the node by (eps, eps^2) in (u, v), i.e. the sign of -(b_v - a_v),    */
/* else of (b_u - a_u).  Each edge and vertex crossing is then counted once */
/* and one ray decides; three rays (+x, +y, +z) vote, so that a node within */
/* rounding of a face (where the "ahead" test t > 0 is decided by rounding) */
/* is still classified by the majority.  Nodes outside the axis-aligned     */
/* bounding box are fluid.                                                  */
/* ------------------------------------------------------------------------- */
static int edge_sign(const double *pa, int ia, const double *pb, int ib, const double P[3], int u, int v) {
  int flip = 1;
  if (ib < ia) { /* canonical order: lower vertex index first */
    const double *t = pa;
    pa = pb;
    pb = t;
    flip = -1;
  }
  double du = pb[u] - pa[u], dv = pb[v] - pa[v];
  double e = du * (P[v] - pa[v]) - dv * (P[u] - pa[u]);
  int sg = e > 0.0 ? 1 : (e < 0.0 ? -1 : 0);
  if (sg == 0) sg = -dv > 0.0 ? 1 : (-dv < 0.0 ? -1 : 0);
  if (sg == 0) sg = du > 0.0 ? 1 : (du < 0.0 ? -1 : 0);
  return flip * sg;
}

static int ray_parity_3d(int ntri, const double *vtx, const int *tri, const double o[3], int axis) {
  const int u = (axis + 1) % 3, v = (axis + 2) % 3;
  int hits = 0;
  for (int f = 0; f < ntri; f++) {
    const int i0 = tri[3 * f], i1 = tri[3 * f + 1], i2 = tri[3 * f + 2];
    const double *a = vtx + 3 * i0, *b = vtx + 3 * i1, *c = vtx + 3 * i2;
    int s0 = edge_sign(a, i0, b, i1, o, u, v);
    int s1 = edge_sign(b, i1, c, i2, o, u, v);
    int s2 = edge_sign(c, i2, a, i0, o, u, v);
    if (s0 == 0 || s0 != s1 || s1 != s2) continue; /* outside the projected triangle (or degenerate edge) */
    /* crossing ahead of the node: t = n.(a - o) / n_axis > 0, n = (b - a) x (c - a) */
    double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    if (n[axis] == 0.0) continue; /* plane parallel to the ray */
    double num = n[0] * (a[0] - o[0]) + n[1] * (a[1] - o[1]) + n[2] * (a[2] - o[2]);
    if ((num > 0.0 && n[axis] > 0.0) || (num < 0.0 && n[axis] < 0.0)) hits++;
  }
  return hits & 1;
}

void orc_classify_points_3d(int nv, const double *verts, int ntri, const int *tris, int np, const double *pts,
                            uint8_t *solid) {
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int k = 0; k < nv; k++)
    for (int a = 0; a < 3; a++) {
      if (verts[3 * k + a] < lo[a]) lo[a] = verts[3 * k + a];
      if (verts[3 * k + a] > hi[a]) hi[a] = verts[3 * k + a];
    }
  for (int n = 0; n < np; n++) {
    const double *o = pts + 3 * n;
    if (o[0] < lo[0] || o[0] > hi[0] || o[1] < lo[1] || o[1] > hi[1] || o[2] < lo[2] || o[2] > hi[2]) {
      solid[n] = 0;
      continue;
    }
    int votes = 0;
    for (int r = 0; r < 3; r++) votes += ray_parity_3d(ntri, verts, tris, o, r);
    solid[n] = (uint8_t)(votes >= 2);
  }
}

/* ------------------------------------------------------------------------- */
/* Sec. 3.2 and Sec. 5, 3-D: node tags from the solid flags of an nx x ny x   */
/* nz lattice (x fastest): IB = fluid node with a solid 6-neighbour; G1..G3 = */
/* solid node whose nearest non-solid node along a grid line is 1, 2 or 3     */
/* nodes away; other solid nodes stay SOLID.                                  */
/* ------------------------------------------------------------------------- */
void orc_tags_3d(int nx, int ny, int nz, const uint8_t *solid, uint8_t *tags) {
  static const int dirs[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
  for (int k = 0; k < nz; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        size_t n = ((size_t)k * ny + j) * nx + i;
        if (!solid[n]) {
          int ib = 0;
          for (int d = 0; d < 6 && !ib; d++) {
            int a = i + dirs[d][0], b = j + dirs[d][1], c = k + dirs[d][2];
            if (a >= 0 && a < nx && b >= 0 && b < ny && c >= 0 && c < nz && solid[((size_t)c * ny + b) * nx + a]) ib = 1;
          }
          tags[n] = ib ? ORC_IB : ORC_FLUID;
          continue;
        }
        tags[n] = ORC_SOLID;
        for (int s = 1; s <= 3; s++) {
          int hit = 0;
          for (int d = 0; d < 6 && !hit; d++) {
            int a = i + s * dirs[d][0], b = j + s * dirs[d][1], c = k + s * dirs[d][2];
            if (a >= 0 && a < nx && b >= 0 && b < ny && c >= 0 && c < nz && !solid[((size_t)c * ny + b) * nx + a])
              hit = 1;
          }
          if (hit) {
            tags[n] = (uint8_t)(ORC_G1 + s - 1);
            break;
          }
        }
      }
}

/* ------------------------------------------------------------------------- */
/* Sec. 4.1-4.2, 3-D: closest feature of a closed triangulated surface and    */
/* its pseudo-normal.  Faces carry their unit normals; a vertex the angle-    */
/* weighted sum of the normals of its faces (Eq. 2); an edge the sum of its   */
/* two faces' normals (Eq. 3, equal weights), all normalised.  The closest    */
/* point on a triangle is the plane projection when it falls inside, else     */
/* the nearest point of the three edges (a vertex when the edge parameter is  */
/* clamped to an end).  The search is exhaustive; ties keep the lowest        */
/* triangle index.  kind: 0 face, 1 edge, 2 vertex.                           */
/* ------------------------------------------------------------------------- */
static void sub3(const double *a, const double *b, double *r) { r[0] = a[0] - b[0]; r[1] = a[1] - b[1]; r[2] = a[2] - b[2]; }
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double *a, const double *b, double *r) {
  r[0] = a[1] * b[2] - a[2] * b[1];
  r[1] = a[2] * b[0] - a[0] * b[2];
  r[2] = a[0] * b[1] - a[1] * b[0];
}
static void unit3(double *a) {
  double L = sqrt(dot3(a, a));
  if (L > 0.0) { a[0] /= L; a[1] /= L; a[2] /= L; }
}

void orc_closest_3d(int nv, const double *v, int ntri, const int *tri, int np, const double *pts, double *cp,
                    double *nrm, int32_t *kind) {
  double *fn = calloc((size_t)3 * ntri, sizeof(double)), *vn = calloc((size_t)3 * nv, sizeof(double));
  /* face normals and angle-weighted vertex sums */
  for (int f = 0; f < ntri; f++) {
    const int *t = tri + 3 * f;
    double e1[3], e2[3];
    sub3(v + 3 * t[1], v + 3 * t[0], e1);
    sub3(v + 3 * t[2], v + 3 * t[0], e2);
    cross3(e1, e2, fn + 3 * f);
    unit3(fn + 3 * f);
    for (int k = 0; k < 3; k++) {
      double a[3], b[3];
      sub3(v + 3 * t[(k + 1) % 3], v + 3 * t[k], a);
      sub3(v + 3 * t[(k + 2) % 3], v + 3 * t[k], b);
      double ang = acos(fmax(-1.0, fmin(1.0, dot3(a, b) / sqrt(dot3(a, a) * dot3(b, b)))));
      for (int d = 0; d < 3; d++) vn[3 * t[k] + d] += ang * fn[3 * f + d];
    }
  }
  for (int k = 0; k < nv; k++) unit3(vn + 3 * k);
  for (int n = 0; n < np; n++) {
    const double *P = pts + 3 * n;
    double best = INFINITY, bc[3] = {0, 0, 0};
    int bf = -1, bk = 0, be = 0, bv = 0;
    for (int f = 0; f < ntri; f++) {
      const int *t = tri + 3 * f;
      const double *A = v + 3 * t[0];
      double e1[3], e2[3], w[3];
      sub3(v + 3 * t[1], A, e1);
      sub3(v + 3 * t[2], A, e2);
      sub3(P, A, w);
      /* plane projection in barycentric form: solve the 2x2 normal equations */
      double a11 = dot3(e1, e1), a12 = dot3(e1, e2), a22 = dot3(e2, e2), b1 = dot3(w, e1), b2 = dot3(w, e2);
      double det = a11 * a22 - a12 * a12;
      double s = (b1 * a22 - b2 * a12) / det, r = (a11 * b2 - a12 * b1) / det;
      double q[3];
      int fk = 0, fe = 0, fv = 0;
      if (s >= 0.0 && r >= 0.0 && s + r <= 1.0) {
        for (int d = 0; d < 3; d++) q[d] = A[d] + s * e1[d] + r * e2[d];
      } else {
        double dmin = INFINITY;
        for (int k = 0; k < 3; k++) {
          const double *E0 = v + 3 * t[k], *E1 = v + 3 * t[(k + 1) % 3];
          double ed[3], pw[3];
          sub3(E1, E0, ed);
          sub3(P, E0, pw);
          double u = dot3(pw, ed) / dot3(ed, ed);
          int vert = -1;
          if (u <= 0.0) { u = 0.0; vert = t[k]; }
          else if (u >= 1.0) { u = 1.0; vert = t[(k + 1) % 3]; }
          double x[3] = {E0[0] + u * ed[0], E0[1] + u * ed[1], E0[2] + u * ed[2]}, dd[3];
          sub3(P, x, dd);
          double d2 = dot3(dd, dd);
          if (d2 < dmin) {
            dmin = d2;
            q[0] = x[0]; q[1] = x[1]; q[2] = x[2];
            fk = vert >= 0 ? 2 : 1;
            fe = k;
            fv = vert;
          }
        }
      }
      double dq[3];
      sub3(P, q, dq);
      double d2 = dot3(dq, dq);
      if (d2 < best) {
        best = d2;
        bf = f; bk = fk; be = fe; bv = fv;
        bc[0] = q[0]; bc[1] = q[1]; bc[2] = q[2];
      }
    }
    double nn[3] = {0, 0, 0};
    if (bk == 0) {
      for (int d = 0; d < 3; d++) nn[d] = fn[3 * bf + d];
    } else if (bk == 2) {
      for (int d = 0; d < 3; d++) nn[d] = vn[3 * bv + d];
    } else {
      /* edge (i, j) of face bf: the neighbouring face holds (j, i) */
      int i = tri[3 * bf + be], j = tri[3 * bf + (be + 1) % 3], g = -1;
      for (int f = 0; f < ntri && g < 0; f++)
        for (int k = 0; k < 3; k++)
          if (tri[3 * f + k] == j && tri[3 * f + (k + 1) % 3] == i) { g = f; break; }
      for (int d = 0; d < 3; d++) nn[d] = fn[3 * bf + d] + (g >= 0 ? fn[3 * g + d] : 0.0);
      unit3(nn);
    }
    for (int d = 0; d < 3; d++) {
      cp[3 * n + d] = bc[d];
      nrm[3 * n + d] = nn[d];
    }
    kind[n] = bk;
  }
  free(fn);
  free(vn);
}

/* ------------------------------------------------------------------------- */
/* Sec. 4.2: pseudo-normals.  Segment k runs from vertex k to k+1 of a CCW   */
/* polyline; its outward normal is the travel direction turned clockwise.    */
/* In 2-D each vertex has two incident segments that enter Eq. 2 with equal  */
/* weight (as the two faces do in Eq. 3), so the vertex pseudo-normal is the */
/* normalised sum of the two adjacent segment normals.                       */
/* ------------------------------------------------------------------------- */
static void build_normals(orc_case *c) {
  int nv = c->p.nv;
  for (int k = 0; k < nv; k++) {
    int k1 = (k + 1 == nv) ? 0 : k + 1;
    double ex = c->vref[2 * k1] - c->vref[2 * k];
    double ey = c->vref[2 * k1 + 1] - c->vref[2 * k + 1];
    double L = sqrt(ex * ex + ey * ey);
    c->snx[k] = ey / L;
    c->sny[k] = -ex / L;
  }
  for (int k = 0; k < nv; k++) {
    int km = (k == 0) ? nv - 1 : k - 1;
    double sx = c->snx[km] + c->snx[k];
    double sy = c->sny[km] + c->sny[k];
    double L = sqrt(sx * sx + sy * sy);
    if (L > 0.0) {
      c->vnx[k] = sx / L;
      c->vny[k] = sy / L;
    } else {
      c->vnx[k] = c->snx[k];
      c->vny[k] = c->sny[k];
    }
  }
  /* Local curvature for the supersonic moving-body condition (Eq. 7): at vertex k the signed Menger curvature */
  /* of (k-1, k, k+1), 2 (e1 x e2) / (|e1| |e2| |e1 + e2|), positive for a left (convex) turn of the CCW      */
  /* polyline; on a regular polygon inscribed in a circle of radius r it is exactly 1/r.                     */
  for (int k = 0; k < nv; k++) {
    int km = (k == 0) ? nv - 1 : k - 1, k1 = (k + 1 == nv) ? 0 : k + 1;
    double e1x = c->vref[2 * k] - c->vref[2 * km], e1y = c->vref[2 * k + 1] - c->vref[2 * km + 1];
    double e2x = c->vref[2 * k1] - c->vref[2 * k], e2y = c->vref[2 * k1 + 1] - c->vref[2 * k + 1];
    double l1 = sqrt(e1x * e1x + e1y * e1y), l2 = sqrt(e2x * e2x + e2y * e2y);
    double sx = e1x + e2x, sy = e1y + e2y;
    double l3 = sqrt(sx * sx + sy * sy);
    double den = l1 * l2 * l3;
    c->vk[k] = den > 0.0 ? 2.0 * (e1x * e2y - e1y * e2x) / den : 0.0;
  }
}

void orc_vertex_normals(const orc_case *c, double *dst) {
  for (int k = 0; k < c->p.nv; k++) {
    dst[2 * k] = c->vnx[k];
    dst[2 * k + 1] = c->vny[k];
  }
}

/* ------------------------------------------------------------------------- */
/* Sec. 4.1: closest surface feature.  Exhaustive search over all segments   */
/* (the bounding-sphere step of the paper only prunes this search).  The     */
/* closest point of a segment is its foot point when that falls strictly     */
/* inside (FACE region), otherwise the nearer end vertex (VERTEX region).    */
/* Ties keep the lowest segment index.                                       */
/* ------------------------------------------------------------------------- */
static void closest_feature(const orc_case *c, double px, double py, int32_t *feat, int32_t *region,
                            double *cxo, double *cyo, double *d2o) {
  int nv = c->p.nv;
  double best = INFINITY;
  for (int k = 0; k < nv; k++) {
    int k1 = (k + 1 == nv) ? 0 : k + 1;
    double ax = c->vx[k], ay = c->vy[k], bx = c->vx[k1], by = c->vy[k1];
    double ex = bx - ax, ey = by - ay;
    double wx = px - ax, wy = py - ay;
    double num = wx * ex + wy * ey;
    double den = ex * ex + ey * ey;
    double cx, cy;
    int32_t f, r;
    if (num <= 0.0) {
      cx = ax; cy = ay; f = k; r = ORC_REGION_VERTEX;
    } else if (num >= den) {
      cx = bx; cy = by; f = k1; r = ORC_REGION_VERTEX;
    } else {
      double t = num / den;
      cx = ax + t * ex; cy = ay + t * ey; f = k; r = ORC_REGION_FACE;
    }
    double ddx = px - cx, ddy = py - cy;
    double d2 = ddx * ddx + ddy * ddy;
    if (d2 < best) {
      best = d2; *feat = f; *region = r; *cxo = cx; *cyo = cy;
    }
  }
  *d2o = best;
}

void orc_closest(const orc_case *c, double px, double py, int32_t *feature, int32_t *region, double *cx,
                 double *cy, double *d2) {
  closest_feature(c, px, py, feature, region, cx, cy, d2);
}

/* ------------------------------------------------------------------------- */
/* Interpolation square and weights around a point (Sec. 4.6, Sec. 5).       */
/* Bilinear when all four corners are valid, otherwise inverse-distance      */
/* weights 1/r^2 over the valid corners; a corner hit exactly takes all the  */
/* weight.  allowed: bit set of tags a corner may carry.                     */
/* ------------------------------------------------------------------------- */
static int interp_square(const orc_case *c, double X, double Y, unsigned allowed, int32_t *i0o, int32_t *j0o,
                         double w[4]) {
  const orc_params *p = &c->p;
  double gx = (X - p->x0) / c->dx - 0.5;
  double gy = (Y - p->y0) / c->dy - 0.5;
  int i0 = (int)floor(gx), j0 = (int)floor(gy);
  int mask = 0;
  for (int k = 0; k < 4; k++) {
    int ci = i0 + (k & 1), cj = j0 + (k >> 1);
    w[k] = 0.0;
    if (ci < 0 || ci >= p->nx || cj < 0 || cj >= p->ny) continue;
    if (allowed & (1u << c->tag[cj * p->nx + ci])) mask |= 1 << k;
  }
  *i0o = i0;
  *j0o = j0;
  if (mask == 15) {
    double xc0 = p->x0 + ((double)i0 + 0.5) * c->dx;
    double yc0 = p->y0 + ((double)j0 + 0.5) * c->dy;
    double fx = (X - xc0) / c->dx;
    double fy = (Y - yc0) / c->dy;
    w[0] = (1.0 - fx) * (1.0 - fy);
    w[1] = fx * (1.0 - fy);
    w[2] = (1.0 - fx) * fy;
    w[3] = fx * fy;
  } else if (mask != 0) {
    double inv[4] = {0, 0, 0, 0};
    double s = 0.0;
    int hit = -1;
    for (int k = 0; k < 4 && hit < 0; k++) {
      if (!(mask >> k & 1)) continue;
      double xk = p->x0 + ((double)(i0 + (k & 1)) + 0.5) * c->dx;
      double yk = p->y0 + ((double)(j0 + (k >> 1)) + 0.5) * c->dy;
      double rx = X - xk, ry = Y - yk;
      double r2 = rx * rx + ry * ry;
      if (r2 == 0.0) hit = k;
      else inv[k] = 1.0 / r2;
    }
    if (hit >= 0) {
      w[hit] = 1.0;
    } else {
      for (int k = 0; k < 4; k++)
        if (mask >> k & 1) s += inv[k];
      for (int k = 0; k < 4; k++)
        if (mask >> k & 1) w[k] = inv[k] / s;
    }
  }
  return mask;
}

/* ------------------------------------------------------------------------- */
/* Sec. 3.2 + Sec. 5: tags and ordered lists.                                */
/*  IB   : fluid node with a solid 4-neighbour (the fluid nodes nearest the  */
/*         surface, Fig. 1); "immediate neighbour" read as the 4-stencil     */
/*         because the flux stencils are axis aligned.                       */
/*  G1-3 : solid node whose nearest non-solid node along a grid line lies k  */
/*         = 1, 2, 3 nodes away (three layers for WENO5, Sec. 5, Fig. 6).    */
/* Lists are in row-major cell order.                                        */
/* ------------------------------------------------------------------------- */
static void build_tags(orc_case *c, const uint8_t *solid) {
  int nx = c->p.nx, ny = c->p.ny;
  static const int DI[4] = {1, -1, 0, 0}, DJ[4] = {0, 0, 1, -1};
  for (int j = 0; j < ny; j++)
    for (int i = 0; i < nx; i++) {
      int n = j * nx + i;
      if (!solid[n]) {
        int ib = 0;
        for (int d = 0; d < 4; d++) {
          int a = i + DI[d], b = j + DJ[d];
          if (a >= 0 && a < nx && b >= 0 && b < ny && solid[b * nx + a]) ib = 1;
        }
        c->tag[n] = ib ? ORC_IB : ORC_FLUID;
      } else {
        int level = 0;
        for (int k = 1; k <= 3 && level == 0; k++)
          for (int d = 0; d < 4; d++) {
            int a = i + k * DI[d], b = j + k * DJ[d];
            if (a >= 0 && a < nx && b >= 0 && b < ny && !solid[b * nx + a]) level = k;
          }
        c->tag[n] = level ? (uint8_t)(ORC_G1 + level - 1) : ORC_SOLID;
      }
    }
}

/* ------------------------------------------------------------------------- */
/* Sec. 4.3: boundary point P' on the line through the node parallel to the  */
/* local normal.  Reading: among the crossings of that line with the         */
/* polyline, take the one nearest the node on the side where the surface     */
/* lies (behind a fluid node, ahead of a ghost node); ties keep the lowest   */
/* segment index.  If the line meets no segment on that side, P' falls back  */
/* to the closest point.  xi_node is the node's signed offset from P' along  */
/* the normal (positive in the fluid).                                       */
/* ------------------------------------------------------------------------- */
static void boundary_point(const orc_case *c, double px, double py, double nx, double ny, int is_ghost,
                           double ccx, double ccy, double *bx, double *by, double *xi_node, int *fallback,
                           int *seg, double *useg) {
  int nv = c->p.nv;
  double best = INFINITY, bs = 0.0, bu = 0.0;
  int found = 0, bk = -1;
  for (int k = 0; k < nv; k++) {
    int k1 = (k + 1 == nv) ? 0 : k + 1;
    double ax = c->vx[k], ay = c->vy[k];
    double ex = c->vx[k1] - ax, ey = c->vy[k1] - ay;
    double den = ex * ny - ey * nx;
    if (den == 0.0) continue;
    double wx = px - ax, wy = py - ay;
    double u = (wx * ny - wy * nx) / den;
    if (u < 0.0 || u > 1.0) continue;
    double s = (wx * ey - wy * ex) / den;
    if (is_ghost ? (s < 0.0) : (s > 0.0)) continue;
    double as = fabs(s);
    if (as < best) {
      best = as; bs = s; bu = u; bk = k; found = 1;
    }
  }
  *seg = bk;
  *useg = bu;
  if (found) {
    *bx = px + bs * nx;
    *by = py + bs * ny;
    *xi_node = -bs;
    *fallback = 0;
  } else {
    double ddx = px - ccx, ddy = py - ccy;
    double d = sqrt(ddx * ddx + ddy * ddy);
    *bx = ccx;
    *by = ccy;
    *xi_node = is_ghost ? -d : d;
    *fallback = 1;
  }
}

/* valid-corner sets: probes of IB nodes and surface probes use fluid nodes,
 * image points of ghost nodes use fluid and (already updated) IB nodes */
#define ALLOW_FLUID (1u << ORC_FLUID)
#define ALLOW_FLUID_IB ((1u << ORC_FLUID) | (1u << ORC_IB))

/* Sec. 4.1-4.6 and Sec. 5: one stencil per listed node. */
static void build_stencil(orc_case *c, int cell, int kind, orc_stencil *s) {
  const orc_params *p = &c->p;
  int i = cell % p->nx, j = cell / p->nx;
  double px = p->x0 + ((double)i + 0.5) * c->dx;
  double py = p->y0 + ((double)j + 0.5) * c->dy;
  int32_t feat = 0, region = 0;
  double ccx = 0, ccy = 0, d2 = 0;
  closest_feature(c, px, py, &feat, &region, &ccx, &ccy, &d2);
  double nx, ny;
  if (region == ORC_REGION_FACE) {
    nx = c->snx[feat]; ny = c->sny[feat];
  } else {
    nx = c->vnx[feat]; ny = c->vny[feat];
  }
  double bx, by, xi_node, useg;
  int fb, seg;
  boundary_point(c, px, py, nx, ny, kind > 0, ccx, ccy, &bx, &by, &xi_node, &fb, &seg, &useg);
  /* curvature at P' (Eq. 7): linear between the end-vertex curvatures of the segment holding P', or the     */
  /* vertex curvature when P' falls back to a closest vertex                                                  */
  double curv;
  if (fb && region == ORC_REGION_VERTEX) {
    curv = c->vk[feat];
  } else {
    if (fb) { /* P' is the foot point on segment feat */
      int k1 = (feat + 1 == p->nv) ? 0 : feat + 1;
      double ex = c->vx[k1] - c->vx[feat], ey = c->vy[k1] - c->vy[feat];
      seg = feat;
      useg = ((ccx - c->vx[feat]) * ex + (ccy - c->vy[feat]) * ey) / (ex * ex + ey * ey);
    }
    int k1 = (seg + 1 == p->nv) ? 0 : seg + 1;
    curv = (1.0 - useg) * c->vk[seg] + useg * c->vk[k1];
  }
  double xi_probe;
  if (kind == 0) {
    xi_probe = xi_node + c->h;              /* probe one diagonal spacing beyond the IB node */
  } else {
    xi_probe = -xi_node;                     /* mirror image point (Fig. 6) */
    if (xi_probe < 0.5 * c->dmin) xi_probe = 0.5 * c->dmin;
  }
  unsigned allowed = kind == 0 ? ALLOW_FLUID : ALLOW_FLUID_IB;
  int32_t i0 = 0, j0 = 0;
  int mask = 0, nstep = 0;
  for (;;) {
    double X = bx + xi_probe * nx, Y = by + xi_probe * ny;
    mask = interp_square(c, X, Y, allowed, &i0, &j0, s->w);
    if (mask != 0 || nstep == 3) break;
    xi_probe = xi_probe + c->dmin;
    nstep++;
  }
  if (mask == 0) c->nerr++;
  s->cell = cell;
  s->feature = feat;
  s->region = fb ? ORC_REGION_FALLBACK : region;
  s->i0 = i0;
  s->j0 = j0;
  s->mask = mask;
  s->nstep = nstep;
  s->kind = kind;
  s->nx = nx;
  s->ny = ny;
  s->bx = bx;
  s->by = by;
  s->xi_node = xi_node;
  s->xi_probe = xi_probe;
  s->curv = curv;
  /* QUADRATIC (Sec. 4.5, Sec. 5): a second probe / image point one diagonal spacing beyond the first, on the   */
  /* same corner set and pushed out the same way while its square has no usable corner                          */
  s->i0b = s->j0b = s->maskb = s->nstepb = 0;
  s->xi_probe2 = 0.0;
  for (int k = 0; k < 4; k++) s->wb[k] = 0.0;
  if (p->ib_interp == ORC_INTERP_QUADRATIC && mask != 0) {
    double xi2 = xi_probe + c->h;
    int32_t ib = 0, jb = 0;
    int maskb = 0, nstepb = 0;
    for (;;) {
      double X = bx + xi2 * nx, Y = by + xi2 * ny;
      maskb = interp_square(c, X, Y, allowed, &ib, &jb, s->wb);
      if (maskb != 0 || nstepb == 3) break;
      xi2 = xi2 + c->dmin;
      nstepb++;
    }
    s->i0b = ib;
    s->j0b = jb;
    s->maskb = maskb;
    s->nstepb = nstepb;
    s->xi_probe2 = xi2;
  }
}

int orc_classify(orc_case *c) {
  const orc_params *p = &c->p;
  int nx = p->nx, ny = p->ny, nc = nx * ny;
  double X[2], V[2], Acc[2];
  motion_at(c, c->t, X, V, Acc);
  c->pos[0] = X[0];
  c->pos[1] = X[1];
  if (p->motion == ORC_MOTION_PITCH) {
    /* rotate the reference pose and its normals about the pivot */
    double th, om, al;
    pitch_at(c, c->t, &th, &om, &al);
    double cs = cos(th), sn = sin(th);
    for (int k = 0; k < p->nv; k++) {
      double rx = c->vref[2 * k] - p->pivot[0], ry = c->vref[2 * k + 1] - p->pivot[1];
      c->vx[k] = p->pivot[0] + (cs * rx - sn * ry);
      c->vy[k] = p->pivot[1] + (sn * rx + cs * ry);
      c->snx[k] = cs * c->snx0[k] - sn * c->sny0[k];
      c->sny[k] = sn * c->snx0[k] + cs * c->sny0[k];
      c->vnx[k] = cs * c->vnx0[k] - sn * c->vny0[k];
      c->vny[k] = sn * c->vnx0[k] + cs * c->vny0[k];
    }
  } else {
    for (int k = 0; k < p->nv; k++) {
      c->vx[k] = c->vref[2 * k] + X[0];
      c->vy[k] = c->vref[2 * k + 1] + X[1];
    }
  }
  uint8_t *solid = calloc(nc, 1);
  if (p->nv > 0) {
    double bb[4];
    bbox(p->nv, c->vx, c->vy, bb);
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        double px = p->x0 + ((double)i + 0.5) * c->dx;
        double py = p->y0 + ((double)j + 0.5) * c->dy;
        solid[j * nx + i] = (uint8_t)point_in_body(p->nv, c->vx, c->vy, bb, px, py);
      }
  }
  build_tags(c, solid);
  free(solid);
  c->nerr = 0;
  for (int kind = 0; kind < 4; kind++) {
    uint8_t want = (uint8_t)(kind == 0 ? ORC_IB : ORC_G1 + kind - 1);
    int n = 0;
    for (int m = 0; m < nc; m++) n += c->tag[m] == want;
    free(c->list[kind]);
    c->list[kind] = calloc(n > 0 ? n : 1, sizeof(orc_stencil));
    c->nlist[kind] = n;
    int w = 0;
    for (int m = 0; m < nc; m++)
      if (c->tag[m] == want) build_stencil(c, m, kind, &c->list[kind][w++]);
  }
  c->classified = 1;
  return c->nerr;
}

/* ------------------------------------------------------------------------- */
/* Primitive variables (Sec. 4.4: the solver works on p, u, v, T).           */
/* ------------------------------------------------------------------------- */
static inline void cons_to_prim(const orc_case *c, double r, double ru, double rv, double rE, double q[4]) {
  double g = c->p.gamma;
  double u = ru / r, v = rv / r;
  double pr = (g - 1.0) * (rE - 0.5 * r * (u * u + v * v));
  q[0] = pr;
  q[1] = u;
  q[2] = v;
  q[3] = pr / (r * c->R);
}

static inline void prim_to_cons(const orc_case *c, const double q[4], double U[4]) {
  double g = c->p.gamma;
  double r = q[0] / (c->R * q[3]);
  U[0] = r;
  U[1] = r * q[1];
  U[2] = r * q[2];
  U[3] = q[0] / (g - 1.0) + 0.5 * r * (q[1] * q[1] + q[2] * q[2]);
}

/* ------------------------------------------------------------------------- */
/* Sec. 4.4-4.6 and Sec. 5: IB and ghost reconstruction at stage time t.     */
/* (ORC_INTERP_QUADRATIC: the quadratic forms in the body of the loop.)      */
/* Velocity is Dirichlet (Eq. 4): linear along the normal through the wall   */
/* value at P' and the interpolated probe value.  Pressure is Neumann        */
/* (Eq. 5-6): dp/dn = -rho n.a_wall; for a body moving faster than sound     */
/* relative to the free stream, the normal force balance of Eq. 7, read in   */
/* the sign convention of Eq. 6: dp/dn = rho u_t^2 / R - rho n.a_wall, with   */
/* u_t the tangential velocity relative to the wall at the probe and 1/R the */
/* stencil's curvature.  Temperature is adiabatic (Eq. 8).  With rho =       */
/* p / (R T) and T fixed along the normal, the pressure condition is a       */
/* linear ODE in p, integrated exactly from the probe to the node.           */
/* IB nodes first (their probes use fluid nodes only), then all ghost layers */
/* (their image points may use the freshly updated IB nodes).                */
/* ------------------------------------------------------------------------- */
static void reconstruct_set(orc_case *c, double *const U[4], const orc_stencil *s, int n, const double Vb[2],
                            const double Ab[2], int supersonic, double t) {
  for (int e = 0; e < n; e++) {
    const orc_stencil *st = &s[e];
    if (st->mask == 0) continue;
    double Vw[2], Aw[2];
    wall_kin(c, t, st->bx, st->by, Vb, Ab, Vw, Aw);  /* the wall's motion at P' */
    double qp[4] = {0, 0, 0, 0};
    for (int k = 0; k < 4; k++) {
      if (!(st->mask >> k & 1)) continue;
      int id = fidx(c, st->i0 + (k & 1), st->j0 + (k >> 1));
      double qk[4];
      cons_to_prim(c, U[0][id], U[1][id], U[2][id], U[3][id], qk);
      for (int v = 0; v < 4; v++) qp[v] += st->w[k] * qk[v];
    }
    double q[4];
    /* dp/dn = rho G with G = -n.a_wall (+ u_t^2 kappa) */
    double G = -(st->nx * Aw[0] + st->ny * Aw[1]);
    if (supersonic) {
      double ut = -(qp[1] - Vw[0]) * st->ny + (qp[2] - Vw[1]) * st->nx;
      G = G + ut * ut * st->curv;
    }
    if (c->p.ib_interp == ORC_INTERP_QUADRATIC && st->maskb != 0) {
      /* the incompressible form (Sec. 4.5, Sec. 5): quadratics in the distance s along the normal through the */
      /* wall condition at P' (s = 0) and the two probes (s1, s2), evaluated at the node (s_n; < 0 for a ghost) */
      double qb[4] = {0, 0, 0, 0};
      for (int k = 0; k < 4; k++) {
        if (!(st->maskb >> k & 1)) continue;
        int id = fidx(c, st->i0b + (k & 1), st->j0b + (k >> 1));
        double qk[4];
        cons_to_prim(c, U[0][id], U[1][id], U[2][id], U[3][id], qk);
        for (int v = 0; v < 4; v++) qb[v] += st->wb[k] * qk[v];
      }
      double s1 = st->xi_probe, s2 = st->xi_probe2, sn = st->xi_node;
      /* velocity, Dirichlet (Eq. 4): Lagrange quadratic through (0, V_w), (s1, q1), (s2, q2) */
      double L1 = sn * (sn - s2) / (s1 * (s1 - s2));
      double L2 = sn * (sn - s1) / (s2 * (s2 - s1));
      q[1] = Vw[0] + (qp[1] - Vw[0]) * L1 + (qb[1] - Vw[0]) * L2;
      q[2] = Vw[1] + (qp[2] - Vw[1]) * L1 + (qb[2] - Vw[1]) * L2;
      /* temperature, adiabatic (Eq. 8), and pressure (Eq. 5-7): a + b s + c s^2 through the two probes with    */
      /* the wall slope b given -- 0, and rho G with the density of the first probe                             */
      double m = (sn * sn - s1 * s1) / (s2 * s2 - s1 * s1);
      double b = qp[0] / (c->R * qp[3]) * G;
      q[3] = qp[3] + (qb[3] - qp[3]) * m;
      q[0] = qp[0] + (qb[0] - qp[0]) * m + b * ((sn - s1) - (s2 - s1) * m);
    } else {
      /* the compressible form: linear through the wall value and the probe for the velocity; T fixed along the */
      /* normal (Eq. 8) and rho = p / (R T), so dp/dn = rho G integrates exactly from the probe to the node:     */
      /* p = p_probe exp(-(xi_p - xi_n) G / (R T))                                                               */
      double ratio = st->xi_node / st->xi_probe;
      q[0] = qp[0] * exp(-(st->xi_probe - st->xi_node) * G / (c->R * qp[3]));
      q[1] = Vw[0] + (qp[1] - Vw[0]) * ratio;
      q[2] = Vw[1] + (qp[2] - Vw[1]) * ratio;
      q[3] = qp[3];
    }
    double Un[4];
    prim_to_cons(c, q, Un);
    int id = fidx(c, st->cell % c->p.nx, st->cell / c->p.nx);
    for (int v = 0; v < 4; v++) U[v][id] = Un[v];
  }
}

/* Eq. 7 applies to a moving body whose speed relative to the free stream exceeds the free-stream sound speed  */
/* (c_inf^2 = gamma p_inf / rho_inf = gamma R).                                                                  */
static int supersonic_motion(const orc_case *c, const double V[2]) {
  if (c->p.motion == ORC_MOTION_STATIC) return 0;
  double rx = V[0] - c->p.uinf[0], ry = V[1] - c->p.uinf[1];
  return rx * rx + ry * ry > c->p.gamma * c->R;
}

static void reconstruct(orc_case *c, double *const U[4], double t) {
  double X[2], V[2], Acc[2];
  motion_at(c, t, X, V, Acc);
  int sup = supersonic_motion(c, V);
  if (c->p.ib_mode != ORC_IB_ADVANCE) reconstruct_set(c, U, c->list[0], c->nlist[0], V, Acc, sup, t);
  for (int k = 1; k < 4; k++) reconstruct_set(c, U, c->list[k], c->nlist[k], V, Acc, sup, t);
}

void orc_reconstruct(orc_case *c, double t) {
  if (!c->classified) orc_classify(c);
  reconstruct(c, c->A, t);
}

/* ------------------------------------------------------------------------- */
/* Domain halos: free-stream Dirichlet, zero-gradient outflow, or periodic.  */
/* y sides first over interior columns, then x sides over all rows.          */
/* ------------------------------------------------------------------------- */
static void domain_bc(orc_case *c, double *const U[4]) {
  const orc_params *p = &c->p;
  int nx = p->nx, ny = p->ny;
  for (int side = 2; side < 4; side++)
    for (int g = 1; g <= NG; g++)
      for (int i = 0; i < nx; i++) {
        int j = side == 2 ? -g : ny - 1 + g;
        int src;
        if (p->bc[side] == ORC_BC_PERIODIC) src = fidx(c, i, side == 2 ? ny - g : g - 1);
        else if (p->bc[side] == ORC_BC_OUTFLOW) src = fidx(c, i, side == 2 ? 0 : ny - 1);
        else src = -1;
        int dst = fidx(c, i, j);
        for (int v = 0; v < 4; v++) U[v][dst] = src < 0 ? c->Uinf[v] : U[v][src];
      }
  for (int side = 0; side < 2; side++)
    for (int g = 1; g <= NG; g++)
      for (int j = -NG; j < ny + NG; j++) {
        int i = side == 0 ? -g : nx - 1 + g;
        int src;
        if (p->bc[side] == ORC_BC_PERIODIC) src = fidx(c, side == 0 ? nx - g : g - 1, j);
        else if (p->bc[side] == ORC_BC_OUTFLOW) src = fidx(c, side == 0 ? 0 : nx - 1, j);
        else src = -1;
        int dst = fidx(c, i, j);
        for (int v = 0; v < 4; v++) U[v][dst] = src < 0 ? c->Uinf[v] : U[v][src];
      }
}

/* ------------------------------------------------------------------------- */
/* Sec. 2: second-order TVD reconstruction (MUSCL with the minmod limiter;   */
/* the paper names the scheme, not its limiter).  f = values at i-1..i+1;    */
/* returns the left-biased value at face i+1/2: f_i + 1/2 minmod of the two  */
/* one-sided differences.                                                    */
/* ------------------------------------------------------------------------- */
double orc_tvd2(const double f[3]) {
  double a = f[1] - f[0], b = f[2] - f[1];
  double m = 0.0;
  if (a > 0.0 && b > 0.0) m = a < b ? a : b;
  else if (a < 0.0 && b < 0.0) m = a > b ? a : b;
  return f[1] + 0.5 * m;
}

/* ------------------------------------------------------------------------- */
/* Sec. 2: fifth-order WENO (Jiang-Shu smoothness indicators, linear weights */
/* 1/10, 6/10, 3/10, eps = 1e-6).  f = values at i-2..i+2; returns the       */
/* left-biased value at face i+1/2.                                          */
/* ------------------------------------------------------------------------- */
double orc_weno5(const double f[5]) {
  const double eps = 1e-6;
  double a = f[0] - 2.0 * f[1] + f[2], b = f[0] - 4.0 * f[1] + 3.0 * f[2];
  double b0 = (13.0 / 12.0) * a * a + 0.25 * b * b;
  a = f[1] - 2.0 * f[2] + f[3];
  b = f[1] - f[3];
  double b1 = (13.0 / 12.0) * a * a + 0.25 * b * b;
  a = f[2] - 2.0 * f[3] + f[4];
  b = 3.0 * f[2] - 4.0 * f[3] + f[4];
  double b2 = (13.0 / 12.0) * a * a + 0.25 * b * b;
  double q0 = (2.0 * f[0] - 7.0 * f[1] + 11.0 * f[2]) / 6.0;
  double q1 = (-f[1] + 5.0 * f[2] + 2.0 * f[3]) / 6.0;
  double q2 = (2.0 * f[2] + 5.0 * f[3] - f[4]) / 6.0;
  double a0 = 0.1 / ((eps + b0) * (eps + b0));
  double a1 = 0.6 / ((eps + b1) * (eps + b1));
  double a2 = 0.3 / ((eps + b2) * (eps + b2));
  return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
}

/* ------------------------------------------------------------------------- */
/* Sec. 2: low-diffusion flux splitting (LDFSS(0) of Edwards) with the       */
/* low-Mach scaled numerical sound speed.  The paper only names the scheme,  */
/* so the reading is:                                                        */
/*   c' = 1/2 sqrt((1 - Mr^2)^2 un^2 + 4 Mr^2 c^2) with face averages,       */
/*   M_L,R = un_L,R / c'; Van Leer splits with the LDFSS pressure-weighted   */
/*   correction; pressure split P+- = (M +- 1)^2 (2 -+ M) / 4.               */
/* mr2 is the face preconditioning parameter Mr^2 (1 = plain LDFSS).        */
/* q = (rho, u, v, p); normal (nxf, nyf) is (1,0) or (0,1).                  */
/* ------------------------------------------------------------------------- */
static void ldfss(const double qL[4], const double qR[4], double nxf, double nyf, double gamma, double R,
                  double cpv, double mr2, double F[4]) {
  (void)R;
  (void)cpv;
  double rL = qL[0], uL = qL[1], vL = qL[2], pL = qL[3];
  double rR = qR[0], uR = qR[1], vR = qR[2], pR = qR[3];
  double cL = sqrt(gamma * pL / rL), cR = sqrt(gamma * pR / rR);
  double HL = gamma / (gamma - 1.0) * pL / rL + 0.5 * (uL * uL + vL * vL);
  double HR = gamma / (gamma - 1.0) * pR / rR + 0.5 * (uR * uR + vR * vR);
  double unL = uL * nxf + vL * nyf, unR = uR * nxf + vR * nyf;
  double cb = 0.5 * (cL + cR);
  double ub = 0.5 * (unL + unR);
  double om = 1.0 - mr2;
  double cs = 0.5 * sqrt(om * om * ub * ub + 4.0 * mr2 * cb * cb);
  double ML = unL / cs, MR = unR / cs;
  double aL = 0.5 * (1.0 + (ML >= 0.0 ? 1.0 : -1.0));
  double aR = 0.5 * (1.0 - (MR >= 0.0 ? 1.0 : -1.0));
  double tL = 1.0 - floor(fabs(ML)), tR = 1.0 - floor(fabs(MR));
  double bL = -(tL > 0.0 ? tL : 0.0), bR = -(tR > 0.0 ? tR : 0.0);
  double MpL = 0.25 * (ML + 1.0) * (ML + 1.0);
  double MmR = -0.25 * (MR - 1.0) * (MR - 1.0);
  double CVL = aL * (1.0 + bL) * ML - bL * MpL;
  double CVR = aR * (1.0 + bR) * MR - bR * MmR;
  double sq = sqrt(0.5 * (ML * ML + MR * MR)) - 1.0;
  double Mh = 0.25 * bL * bR * sq * sq;
  double dp = pL - pR, adp = fabs(dp);
  double MhP = Mh * (1.0 - (dp + adp) / (2.0 * rL * cs * cs));
  double MhM = Mh * (1.0 - (-dp + adp) / (2.0 * rR * cs * cs));
  double Cp = CVL - MhP, Cm = CVR + MhM;
  /* pressure split with the physical face Mach numbers un/c.  With low-Mach scaling (mr2 < 1) its        */
  /* dissipative part -- the departure of D_L p_L + D_R p_R from the face mean, about (3/4) rho c (uL - uR) */
  /* at low Mach -- is scaled by fa = c'/c, so that it acts like rho c' (uL - uR) with c' of the order of  */
  /* the flow speed (reading: the paper only names the scheme; the unscaled split keeps O(M) pressure     */
  /* fluctuations and loses the incompressible limit, the split in the scaled Mach numbers un/c' raises   */
  /* that term by c/c' and made the pseudo-time iteration diverge).  mr2 = 1 gives plain LDFSS(0).        */
  double pL_ = ML, pR_ = MR, paL = aL, paR = aR, pbL = bL, pbR = bR;
  if (mr2 < 1.0) {
    pL_ = unL / cb;
    pR_ = unR / cb;
    paL = 0.5 * (1.0 + (pL_ >= 0.0 ? 1.0 : -1.0));
    paR = 0.5 * (1.0 - (pR_ >= 0.0 ? 1.0 : -1.0));
    double uL_ = 1.0 - floor(fabs(pL_)), uR_ = 1.0 - floor(fabs(pR_));
    pbL = -(uL_ > 0.0 ? uL_ : 0.0);
    pbR = -(uR_ > 0.0 ? uR_ : 0.0);
  }
  double PpL = 0.25 * (pL_ + 1.0) * (pL_ + 1.0) * (2.0 - pL_);
  double PmR = 0.25 * (pR_ - 1.0) * (pR_ - 1.0) * (2.0 + pR_);
  double DL = paL * (1.0 + pbL) - pbL * PpL;
  double DR = paR * (1.0 + pbR) - pbR * PmR;
  double mL = rL * cs * Cp, mR = rR * cs * Cm;
  double ph = DL * pL + DR * pR;
  if (mr2 < 1.0) {
    double fa = cs / cb;
    ph = 0.5 * (pL + pR) + fa * ((DL - 0.5) * pL + (DR - 0.5) * pR);
  }
  F[0] = mL + mR;
  F[1] = mL * uL + mR * uR + ph * nxf;
  F[2] = mL * vL + mR * vR + ph * nyf;
  F[3] = mL * HL + mR * HR;
}

void orc_ldfss_xflux(const double qL[4], const double qR[4], double gamma, double R, double mr2_fixed,
                     double flux[4]) {
  double cpv = gamma * R / (gamma - 1.0);
  ldfss(qL, qR, 1.0, 0.0, gamma, R, cpv, mr2_fixed, flux);
}

void orc_euler_xflux(const double q[4], double gamma, double R, double flux[4]) {
  (void)R;
  double r = q[0], u = q[1], v = q[2], p = q[3];
  double H = gamma / (gamma - 1.0) * p / r + 0.5 * (u * u + v * v);
  flux[0] = r * u;
  flux[1] = r * u * u + p;
  flux[2] = r * u * v;
  flux[3] = r * u * H;
}

/* Low-Mach preconditioning parameter at a face.  Only the dual-time scheme,
 * whose pseudo-time derivative carries the preconditioning matrix, scales the
 * dissipation; explicit physical-time stepping uses plain LDFSS (Mr^2 = 1).
 * Reference velocity Ur = min(c, max(|V|, U_ref, nu/dn)), Mr^2 = (Ur/c)^2
 * with face-averaged c, |V| and rho (Weiss-Smith; no lower bound tied to c,
 * so that the dissipation follows the flow speed as M -> 0). */
static double face_mr2(const orc_case *c, const double qL[4], const double qR[4], double dn) {
  if (!c->precond) return 1.0;
  double g = c->p.gamma;
  double cb = 0.5 * (sqrt(g * qL[3] / qL[0]) + sqrt(g * qR[3] / qR[0]));
  double ub = 0.5 * (qL[1] + qR[1]), vb = 0.5 * (qL[2] + qR[2]);
  double Vm = sqrt(ub * ub + vb * vb);
  double rb = 0.5 * (qL[0] + qR[0]);
  double vis = c->mu / rb / dn;
  double Ur = Vm;
  if (1.0 > Ur) Ur = 1.0;
  if (vis > Ur) Ur = vis;
  if (cb < Ur) Ur = cb;
  double m = (Ur / cb) * (Ur / cb);
  return m < 1.0 ? m : 1.0;
}

/* WENO5 left/right states of the reconstructed primitives (rho, u, v, p) at
 * the face between cells s[2] and s[3] of the six-cell strip s[0..5]; first-
 * order fallback if a reconstructed density or pressure is not positive.
 * Reading: the paper iterates (p, u, v, w, T) but does not say which set WENO
 * acts on; (rho, u, v, p) keeps a density wave at fifth order because every
 * flux component is affine in rho when u and p are uniform. */
static void face_states(const orc_case *c, const double s[6][4], double qL[4], double qR[4]) {
  for (int v = 0; v < 4; v++) {
    if (c->p.scheme == ORC_SCHEME_TVD2) {
      double fl[3] = {s[1][v], s[2][v], s[3][v]};
      double fr[3] = {s[4][v], s[3][v], s[2][v]};
      qL[v] = orc_tvd2(fl);
      qR[v] = orc_tvd2(fr);
      continue;
    }
    double fl[5] = {s[0][v], s[1][v], s[2][v], s[3][v], s[4][v]};
    double fr[5] = {s[5][v], s[4][v], s[3][v], s[2][v], s[1][v]};
    qL[v] = orc_weno5(fl);
    qR[v] = orc_weno5(fr);
  }
  if (!(qL[0] > 0.0) || !(qL[3] > 0.0) || !(qR[0] > 0.0) || !(qR[3] > 0.0)) {
    for (int v = 0; v < 4; v++) {
      qL[v] = s[2][v];
      qR[v] = s[3][v];
    }
  }
}

/* Sec. 2: residual L(U) = -(dF/dx + dG/dy) over fluid cells, inviscid
 * (WENO5 + LDFSS) minus viscous (second-order central) face fluxes. */
static void residual_faces(orc_case *c, double *const U[4]) {
  const orc_params *p = &c->p;
  int nx = p->nx, ny = p->ny, W = c->W, H = c->H;
  double g = p->gamma, R = c->R, mu = c->mu, kap = c->kappa, cpv = c->cp;
  for (int m = 0; m < W * H; m++) {
    double r = U[0][m], u = U[1][m] / r, v = U[2][m] / r;
    double pr = (g - 1.0) * (U[3][m] - 0.5 * r * (u * u + v * v));
    c->q[0][m] = r;
    c->q[1][m] = u;
    c->q[2][m] = v;
    c->q[3][m] = pr;
    c->T[m] = pr / (r * R);
  }
  double *const *Q = c->q;
  /* x-faces: face f = i + 1/2 for i in [-1, nx-1], stored at fidx(i, j) */
#pragma omp parallel for schedule(static)
  for (int j = 0; j < ny; j++)
    for (int i = -1; i < nx; i++) {
      double s[6][4];
      for (int k = 0; k < 6; k++)
        for (int v = 0; v < 4; v++) s[k][v] = Q[v][fidx(c, i - 2 + k, j)];
      double qL[4], qR[4], F[4];
      face_states(c, s, qL, qR);
      ldfss(qL, qR, 1.0, 0.0, g, R, cpv, face_mr2(c, qL, qR, c->dx), F);
      int a = fidx(c, i, j), b = fidx(c, i + 1, j);
      int an = fidx(c, i, j + 1), as = fidx(c, i, j - 1), bn = fidx(c, i + 1, j + 1), bs = fidx(c, i + 1, j - 1);
      double ux = (Q[1][b] - Q[1][a]) / c->dx, vx = (Q[2][b] - Q[2][a]) / c->dx, Tx = (c->T[b] - c->T[a]) / c->dx;
      double uy = (Q[1][an] - Q[1][as] + Q[1][bn] - Q[1][bs]) / (4.0 * c->dy);
      double vy = (Q[2][an] - Q[2][as] + Q[2][bn] - Q[2][bs]) / (4.0 * c->dy);
      double txx = mu * ((4.0 / 3.0) * ux - (2.0 / 3.0) * vy);
      double txy = mu * (uy + vx);
      double qx = -kap * Tx;
      double uf = 0.5 * (Q[1][a] + Q[1][b]), vf = 0.5 * (Q[2][a] + Q[2][b]);
      c->fx[0][a] = F[0];
      c->fx[1][a] = F[1] - txx;
      c->fx[2][a] = F[2] - txy;
      c->fx[3][a] = F[3] - (uf * txx + vf * txy - qx);
    }
  /* y-faces: face j + 1/2 for j in [-1, ny-1], stored at fidx(i, j) */
#pragma omp parallel for schedule(static)
  for (int j = -1; j < ny; j++)
    for (int i = 0; i < nx; i++) {
      double s[6][4];
      for (int k = 0; k < 6; k++)
        for (int v = 0; v < 4; v++) s[k][v] = Q[v][fidx(c, i, j - 2 + k)];
      double qL[4], qR[4], F[4];
      face_states(c, s, qL, qR);
      ldfss(qL, qR, 0.0, 1.0, g, R, cpv, face_mr2(c, qL, qR, c->dy), F);
      int a = fidx(c, i, j), b = fidx(c, i, j + 1);
      int ae = fidx(c, i + 1, j), aw = fidx(c, i - 1, j), be = fidx(c, i + 1, j + 1), bw = fidx(c, i - 1, j + 1);
      double uy = (Q[1][b] - Q[1][a]) / c->dy, vy = (Q[2][b] - Q[2][a]) / c->dy, Ty = (c->T[b] - c->T[a]) / c->dy;
      double ux = (Q[1][ae] - Q[1][aw] + Q[1][be] - Q[1][bw]) / (4.0 * c->dx);
      double vx = (Q[2][ae] - Q[2][aw] + Q[2][be] - Q[2][bw]) / (4.0 * c->dx);
      double tyy = mu * ((4.0 / 3.0) * vy - (2.0 / 3.0) * ux);
      double txy = mu * (uy + vx);
      double qy = -kap * Ty;
      double uf = 0.5 * (Q[1][a] + Q[1][b]), vf = 0.5 * (Q[2][a] + Q[2][b]);
      c->fy[0][a] = F[0];
      c->fy[1][a] = F[1] - txy;
      c->fy[2][a] = F[2] - tyy;
      c->fy[3][a] = F[3] - (uf * txy + vf * tyy - qy);
    }
}

/* SSP-RK3 (Shu-Osher) stage on fluid cells:
 *   stage 1: out = Un + dt L(in)
 *   stage 2: out = 3/4 Un + 1/4 (in + dt L(in))
 *   stage 3: out = 1/3 Un + 2/3 (in + dt L(in)) */
static void stage_update(orc_case *c, int stage, double *const Un[4], double *const In[4], double *const Out[4],
                         double dt) {
  const orc_params *p = &c->p;
  int nx = p->nx, ny = p->ny;
#pragma omp parallel for schedule(static)
  for (int j = 0; j < ny; j++)
    for (int i = 0; i < nx; i++) {
      if (!advanced(c, c->tag[j * nx + i])) continue;
      int m = fidx(c, i, j), mw = fidx(c, i - 1, j), ms = fidx(c, i, j - 1);
      for (int v = 0; v < 4; v++) {
        double L = -((c->fx[v][m] - c->fx[v][mw]) / c->dx + (c->fy[v][m] - c->fy[v][ms]) / c->dy);
        double o;
        if (stage == 1) o = Un[v][m] + dt * L;
        else if (stage == 2) o = 0.75 * Un[v][m] + 0.25 * (In[v][m] + dt * L);
        else o = (1.0 / 3.0) * Un[v][m] + (2.0 / 3.0) * (In[v][m] + dt * L);
        Out[v][m] = o;
      }
    }
}

/* Time step from the CFL rule over fluid cells:
 * dt = CFL / max[(|u|+c)/dx + (|v|+c)/dy + 2 gamma mu/(Pr rho) (1/dx^2 + 1/dy^2)]. */
static double compute_dt(orc_case *c) {
  const orc_params *p = &c->p;
  if (p->dt_fixed > 0.0) return p->dt_fixed;
  double lmax = 0.0, g = p->gamma;
  for (int j = 0; j < p->ny; j++)
    for (int i = 0; i < p->nx; i++) {
      if (!advanced(c, c->tag[j * p->nx + i])) continue;
      int m = fidx(c, i, j);
      double q[4];
      cons_to_prim(c, c->A[0][m], c->A[1][m], c->A[2][m], c->A[3][m], q);
      double cs = sqrt(g * c->R * q[3]);
      double rho = c->A[0][m];
      double lam = (fabs(q[1]) + cs) / c->dx + (fabs(q[2]) + cs) / c->dy +
                   (2.0 * g * c->mu / (p->prandtl * rho)) * (1.0 / (c->dx * c->dx) + 1.0 / (c->dy * c->dy));
      if (lam > lmax) lmax = lam;
    }
  return p->cfl / lmax;
}

/* ------------------------------------------------------------------------- */
/* Dual time stepping (Sec. 2): three-point (BDF2) physical-time derivative,  */
/* two-point Euler pseudo-time derivative with the low-Mach preconditioning   */
/* matrix, point-implicit in the physical-time term.  The increment of one   */
/* pseudo step, for each fluid cell,                                         */
/*   [Gamma/dtau + (3/(2 dt)) dW/dQ] dQ = -( R(W) + (3W - 4W^n + W^{n-1})/(2 dt) )      */
/* is applied as the three stages of SSP-RK3 in Q (reading: a single forward  */
/* Euler pseudo step diverges at low Mach, where the physical-time term does  */
/* not damp the preconditioned acoustic mode); one sub-iteration = one such  */
/* three-stage pseudo step.                                                  */
/* (first physical step: BDF1, (1/dt) dW/dQ and (W^k - W^n)/dt), with        */
/* R = dF/dx + dG/dy the residual (preconditioned LDFSS dissipation).  The    */
/* paper names the scheme only; the matrix is the Weiss-Smith form in        */
/* primitive variables Q = (p, u, v, T):                                     */
/*   rows [T, 0, 0, rT], [T u, r, 0, rT u], [T v, 0, r, rT v],                */
/*        [T H - 1, r u, r v, rT H + r cp]                                   */
/* with rT = -r/T and T = 1/Ur^2 - rT/(r cp) (Gamma) or 1/(R T) (dW/dQ).       */
/* Ur = min(c, max(|V|, U_ref, nu/dmin)); local dtau = CFL_tau / [(|u'|+c') */
/* (1/dx + 1/dy) + 2 gamma mu/(Pr r)(1/dx^2 + 1/dy^2)], u', c' the           */
/* eigenvalue terms of the preconditioned system.  The 4x4 system is solved  */
/* by Gaussian elimination with partial pivoting.                            */
/* ------------------------------------------------------------------------- */
static void wq_matrix(double theta, const double Q[4], double gamma, double R, double M[16]) {
  double p = Q[0], u = Q[1], v = Q[2], T = Q[3];
  double r = p / (R * T);
  double cpv = gamma * R / (gamma - 1.0);
  double rT = -r / T;
  double H = cpv * T + 0.5 * (u * u + v * v);
  double row[16] = {theta,           0.0,   0.0,   rT,
                    theta * u,       r,     0.0,   rT * u,
                    theta * v,       0.0,   r,     rT * v,
                    theta * H - 1.0, r * u, r * v, rT * H + r * cpv};
  for (int i = 0; i < 16; i++) M[i] = row[i];
}

void orc_precond_matrix(const double Q[4], double gamma, double R, double Ur, double out[16]) {
  double r = Q[0] / (R * Q[3]);
  double cpv = gamma * R / (gamma - 1.0);
  double theta = 1.0 / (Ur * Ur) - (-r / Q[3]) / (r * cpv);
  wq_matrix(theta, Q, gamma, R, out);
}

void orc_dwdq(const double Q[4], double gamma, double R, double out[16]) {
  wq_matrix(1.0 / (R * Q[3]), Q, gamma, R, out);
}

int orc_solve4(const double Ain[16], const double bin[4], double x[4]) {
  double A[4][5];
  for (int i = 0; i < 4; i++) {
    for (int j = 0; j < 4; j++) A[i][j] = Ain[4 * i + j];
    A[i][4] = bin[i];
  }
  for (int col = 0; col < 4; col++) {
    int piv = col;
    for (int i = col + 1; i < 4; i++)
      if (fabs(A[i][col]) > fabs(A[piv][col])) piv = i;
    if (A[piv][col] == 0.0) return -1;
    if (piv != col)
      for (int j = 0; j < 5; j++) {
        double t = A[col][j];
        A[col][j] = A[piv][j];
        A[piv][j] = t;
      }
    for (int i = col + 1; i < 4; i++) {
      double f = A[i][col] / A[col][col];
      for (int j = col; j < 5; j++) A[i][j] -= f * A[col][j];
    }
  }
  for (int i = 3; i >= 0; i--) {
    double s = A[i][4];
    for (int j = i + 1; j < 4; j++) s -= A[i][j] * x[j];
    x[i] = s / A[i][i];
  }
  return 0;
}

static void dual_update(orc_case *c, int stage, double *const In[4], double *const Out[4], int bdf2) {
  const orc_params *p = &c->p;
  int nx = p->nx, ny = p->ny;
  double g = p->gamma, R = c->R, dt = p->dt_phys;
  double vis = (2.0 * g * c->mu / p->prandtl) * (1.0 / (c->dx * c->dx) + 1.0 / (c->dy * c->dy));
#pragma omp parallel for schedule(static)
  for (int j = 0; j < ny; j++)
    for (int i = 0; i < nx; i++) {
      if (!advanced(c, c->tag[j * nx + i])) continue;
      int m = fidx(c, i, j), mw = fidx(c, i - 1, j), ms = fidx(c, i, j - 1);
      double W[4], Q[4], S[4];
      for (int v = 0; v < 4; v++) W[v] = In[v][m];
      cons_to_prim(c, W[0], W[1], W[2], W[3], Q);
      for (int v = 0; v < 4; v++) {
        double Rv = (c->fx[v][m] - c->fx[v][mw]) / c->dx + (c->fy[v][m] - c->fy[v][ms]) / c->dy;
        double tdt = bdf2 ? (3.0 * W[v] - 4.0 * c->Wn[v][m] + c->Wm[v][m]) / (2.0 * dt) : (W[v] - c->Wn[v][m]) / dt;
        S[v] = -(Rv + tdt);
      }
      double r = W[0];
      double cs = sqrt(g * Q[0] / r);
      double Vm = sqrt(Q[1] * Q[1] + Q[2] * Q[2]);
      double Ur = Vm;
      if (1.0 > Ur) Ur = 1.0;
      if (c->mu / r / c->dmin > Ur) Ur = c->mu / r / c->dmin;
      if (cs < Ur) Ur = cs;
      double mr2 = (Ur / cs) * (Ur / cs);
      double up = 0.5 * Vm * (1.0 + mr2);
      double om = 1.0 - mr2;
      double cp_ = 0.5 * sqrt(om * om * Vm * Vm + 4.0 * Ur * Ur);
      double lam = (up + cp_) * (1.0 / c->dx + 1.0 / c->dy) + vis / r;
      double dtau = p->cfl_tau / lam;
      double G[16], J[16], M[16], dQ[4];
      orc_precond_matrix(Q, g, R, Ur, G);
      orc_dwdq(Q, g, R, J);
      double a = bdf2 ? 1.5 / dt : 1.0 / dt;
      for (int q = 0; q < 16; q++) M[q] = G[q] / dtau + a * J[q];
      if (orc_solve4(M, S, dQ) != 0) continue;
      /* SSP-RK3 combination in Q with the sub-iteration's starting iterate Q0 (held in A) */
      double Q0[4], Qn[4];
      cons_to_prim(c, c->A[0][m], c->A[1][m], c->A[2][m], c->A[3][m], Q0);
      for (int v = 0; v < 4; v++) {
        double e = Q[v] + dQ[v];
        if (stage == 1) Qn[v] = e;
        else if (stage == 2) Qn[v] = 0.75 * Q0[v] + 0.25 * e;
        else Qn[v] = (1.0 / 3.0) * Q0[v] + (2.0 / 3.0) * e;
      }
      double Un[4];
      prim_to_cons(c, Qn, Un);
      for (int v = 0; v < 4; v++) Out[v][m] = Un[v];
    }
}

static void dual_step(orc_case *c) {
  if (!c->classified || c->p.motion != ORC_MOTION_STATIC) orc_classify(c);
  const orc_params *p = &c->p;
  size_t n = (size_t)c->W * c->H;
  for (int v = 0; v < 4; v++) {
    if (c->nphys > 0) memcpy(c->Wm[v], c->Wn[v], n * sizeof(double));
    memcpy(c->Wn[v], c->A[v], n * sizeof(double));
  }
  int bdf2 = c->nphys > 0;
  double t1 = c->t + p->dt_phys;
  double *const *in[3] = {c->A, c->B, c->C};
  double *const *out[3] = {c->B, c->C, c->A};
  for (int k = 0; k < p->subiters; k++)
    for (int st = 0; st < 3; st++) {
      reconstruct(c, in[st], t1);
      domain_bc(c, in[st]);
      residual_faces(c, in[st]);
      dual_update(c, st + 1, in[st], out[st], bdf2);
    }
  (void)n;
  c->t = t1;
  c->last_dt = p->dt_phys;
  c->nphys++;
}

int orc_step(orc_case *c, int nsteps) {
  if (c->p.time_scheme == ORC_TIME_DUAL) {
    for (int s = 0; s < nsteps; s++) dual_step(c);
    return c->nerr;
  }
  for (int s = 0; s < nsteps; s++) {
    if (!c->classified || c->p.motion != ORC_MOTION_STATIC) orc_classify(c);
    if (c->p.motion == ORC_MOTION_COUPLED) {
      /* Eq. 10: the force on the body at t^n (its wall pressure carried with the previous acceleration) */
      /* sets the acceleration of the step                                                                */
      double f[4];
      orc_forces(c, f);
      for (int k = 0; k < 2; k++) {
        c->bF[k] = f[2 + k];
        c->bA[k] = f[2 + k] / c->p.mass;
      }
    }
    double dt = compute_dt(c);
    double t = c->t;
    double ts[3] = {t, t + dt, t + 0.5 * dt};
    double *const *in[3] = {c->A, c->B, c->C};
    double *const *out[3] = {c->B, c->C, c->A};
    for (int k = 0; k < 3; k++) {
      reconstruct(c, in[k], ts[k]);
      domain_bc(c, in[k]);
      residual_faces(c, in[k]);
      stage_update(c, k + 1, c->A, in[k], out[k], dt);
    }
    c->t = t + dt;
    c->last_dt = dt;
    if (c->p.motion == ORC_MOTION_COUPLED) {
      /* Eq. 10 with the position advanced by the constant-acceleration step (the printed update lacks the */
      /* factor 1/2 of the step's (dt)^2 term): x += U dt + dt^2 F / (2 M), U += dt F / M                   */
      for (int k = 0; k < 2; k++) {
        c->bX[k] = c->bX[k] + dt * c->bV[k] + 0.5 * dt * dt * c->bA[k];
        c->bV[k] = c->bV[k] + dt * c->bA[k];
      }
      c->bt = c->t;
    }
  }
  return c->nerr;
}

void orc_body(const orc_case *c, double out[6]) {
  for (int k = 0; k < 2; k++) {
    out[k] = c->bX[k];
    out[2 + k] = c->bV[k];
    out[4 + k] = c->bF[k];
  }
}

/* ------------------------------------------------------------------------- */
/* Sec. 6, Eq. 9: force on the body.  Midpoint rule per segment; surface     */
/* pressure and wall shear from the probe one diagonal spacing out along the */
/* segment normal (inverse-distance weighted as in Sec. 4.6); the pressure  */
/* is carried to the wall by the wall condition of the reconstruction (Eq.   */
/* 6-8, curvature at the segment midpoint = mean of its vertex values).     */
/* The free-stream pressure is subtracted (its closed-surface integral is   */
/* zero).                                                                    */
/* Compensated (Kahan) summation.                                            */
/* ------------------------------------------------------------------------- */
/* Eq. 9 integrand on segment k: unit tangent and normal, length, wall      */
/* pressure ps and wall shear tau at the midpoint.  Returns 0 when no probe */
/* square is found (the segment is then left out of the sums).             */
static int surface_segment(orc_case *c, int k, const double V[2], const double Acc[2], int sup, double *ps_o,
                           double *tau_o, double *L_o, double *tx_o, double *ty_o) {
  const orc_params *p = &c->p;
  int k1 = (k + 1 == p->nv) ? 0 : k + 1;
  double ax = c->vx[k], ay = c->vy[k];
  double ex = c->vx[k1] - ax, ey = c->vy[k1] - ay;
  double L = sqrt(ex * ex + ey * ey);
  double tx = ex / L, ty = ey / L;
  double nx = ty, ny = -tx;
  double mx = ax + 0.5 * ex, my = ay + 0.5 * ey;
  double xi = c->h, w[4];
  int32_t i0, j0;
  int mask = 0;
  for (int st = 0; st <= 3; st++) {
    mask = interp_square(c, mx + xi * nx, my + xi * ny, ALLOW_FLUID, &i0, &j0, w);
    if (mask) break;
    if (st < 3) xi = xi + c->dmin;
  }
  if (!mask) return 0;
  double qp[4] = {0, 0, 0, 0};
  for (int kk = 0; kk < 4; kk++) {
    if (!(mask >> kk & 1)) continue;
    int id = fidx(c, i0 + (kk & 1), j0 + (kk >> 1));
    double qk[4];
    cons_to_prim(c, c->A[0][id], c->A[1][id], c->A[2][id], c->A[3][id], qk);
    for (int v = 0; v < 4; v++) qp[v] += w[kk] * qk[v];
  }
  /* wall pressure: the probe's, carried to the surface by the wall condition of the reconstruction */
  double Vs[2], As[2];
  wall_kin(c, c->t, mx, my, V, Acc, Vs, As);  /* the wall's motion at the segment midpoint */
  double G = -(nx * As[0] + ny * As[1]);
  if (sup) {
    double ut = (qp[1] - Vs[0]) * tx + (qp[2] - Vs[1]) * ty;
    G = G + ut * ut * (0.5 * (c->vk[k] + c->vk[k1]));
  }
  /* wall shear: the tangential velocity relative to the wall over the probe distance */
  *ps_o = qp[0] * exp(-xi * G / (c->R * qp[3]));
  *tau_o = c->mu * ((qp[1] - Vs[0]) * tx + (qp[2] - Vs[1]) * ty) / xi;
  *L_o = L;
  *tx_o = tx;
  *ty_o = ty;
  return 1;
}

void orc_forces(orc_case *c, double out[4]) {
  const orc_params *p = &c->p;
  if (!c->classified) orc_classify(c);
  double X[2], V[2], Acc[2];
  motion_at(c, c->t, X, V, Acc);
  int sup = supersonic_motion(c, V);
  double sx = 0, cx = 0, sy = 0, cy = 0;
  for (int k = 0; k < p->nv; k++) {
    double ps, tau, L, tx, ty;
    if (!surface_segment(c, k, V, Acc, sup, &ps, &tau, &L, &tx, &ty)) continue;
    double nx = ty, ny = -tx;
    double fx = (-(ps - c->pinf) * nx + tau * tx) * L;
    double fy = (-(ps - c->pinf) * ny + tau * ty) * L;
    double y1 = fx - cx, t1 = sx + y1;
    cx = (t1 - sx) - y1;
    sx = t1;
    double y2 = fy - cy, t2 = sy + y2;
    cy = (t2 - sy) - y2;
    sy = t2;
  }
  double qref = 0.5 * p->ref_len;
  out[0] = sx / qref;
  out[1] = sy / qref;
  out[2] = sx;
  out[3] = sy;
}

/* Surface distributions of Eq. 9 per segment: pressure coefficient       */
/* (ps - p_inf) / (rho_inf U^2 / 2) and skin-friction coefficient          */
/* tau / (rho_inf U^2 / 2) at the segment midpoints; NaN where no probe.   */
void orc_surface(orc_case *c, double *cp, double *cf) {
  const orc_params *p = &c->p;
  if (!c->classified) orc_classify(c);
  double X[2], V[2], Acc[2];
  motion_at(c, c->t, X, V, Acc);
  int sup = supersonic_motion(c, V);
  for (int k = 0; k < p->nv; k++) {
    double ps, tau, L, tx, ty;
    if (!surface_segment(c, k, V, Acc, sup, &ps, &tau, &L, &tx, &ty)) {
      cp[k] = NAN;
      cf[k] = NAN;
      continue;
    }
    cp[k] = (ps - c->pinf) / 0.5;
    cf[k] = tau / 0.5;
  }
}

/* ------------------------------------------------------------------------- */
/* setup.  Non-dimensional free stream: rho = 1, T = 1, reference speed 1,    */
/* p = 1/(gamma M^2), R = p, mu = 1/Re (reference length 1), k = mu cp / Pr. */
/* ------------------------------------------------------------------------- */
orc_case *orc_create(const orc_params *pp) {
  orc_case *c = calloc(1, sizeof(orc_case));
  c->p = *pp;
  const orc_params *p = &c->p;
  int nv = p->nv;
  c->vref = calloc(2 * (nv > 0 ? nv : 1), sizeof(double));
  if (nv > 0) memcpy(c->vref, pp->verts, sizeof(double) * 2 * nv);
  c->p.verts = c->vref;
  c->vx = calloc(nv > 0 ? nv : 1, sizeof(double));
  c->vy = calloc(nv > 0 ? nv : 1, sizeof(double));
  c->snx = calloc(nv > 0 ? nv : 1, sizeof(double));
  c->sny = calloc(nv > 0 ? nv : 1, sizeof(double));
  c->vnx = calloc(nv > 0 ? nv : 1, sizeof(double));
  c->vny = calloc(nv > 0 ? nv : 1, sizeof(double));
  c->vk = calloc(nv > 0 ? nv : 1, sizeof(double));
  if (nv > 0) build_normals(c);
  if (nv > 0 && p->motion == ORC_MOTION_PITCH) {  /* reference normals, rotated at every classification */
    c->snx0 = malloc(nv * sizeof(double));
    c->sny0 = malloc(nv * sizeof(double));
    c->vnx0 = malloc(nv * sizeof(double));
    c->vny0 = malloc(nv * sizeof(double));
    memcpy(c->snx0, c->snx, nv * sizeof(double));
    memcpy(c->sny0, c->sny, nv * sizeof(double));
    memcpy(c->vnx0, c->vnx, nv * sizeof(double));
    memcpy(c->vny0, c->vny, nv * sizeof(double));
  }
  {
    double X[2], V[2], Acc[2];
    for (int k = 0; k < 2; k++) {
      c->bX[k] = 0.0;
      c->bV[k] = p->motion == ORC_MOTION_COUPLED ? p->vel[k] : 0.0;
      c->bA[k] = c->bF[k] = 0.0;
    }
    c->bt = 0.0;
    motion_at(c, 0.0, X, V, Acc);
    for (int k = 0; k < nv; k++) {
      c->vx[k] = c->vref[2 * k] + X[0];
      c->vy[k] = c->vref[2 * k + 1] + X[1];
    }
  }
  c->dx = (p->x1 - p->x0) / p->nx;
  c->dy = (p->y1 - p->y0) / p->ny;
  c->h = sqrt(c->dx * c->dx + c->dy * c->dy);
  c->dmin = c->dx < c->dy ? c->dx : c->dy;
  double g = p->gamma;
  c->pinf = 1.0 / (g * p->mach * p->mach);
  c->R = c->pinf;
  c->cp = g * c->R / (g - 1.0);
  c->mu = p->re > 0.0 ? 1.0 / p->re : 0.0;
  c->kappa = c->mu * c->cp / p->prandtl;
  c->Uinf[0] = 1.0;
  c->Uinf[1] = p->uinf[0];
  c->Uinf[2] = p->uinf[1];
  c->Uinf[3] = c->pinf / (g - 1.0) + 0.5 * (p->uinf[0] * p->uinf[0] + p->uinf[1] * p->uinf[1]);
  c->W = p->nx + 2 * NG;
  c->H = p->ny + 2 * NG;
  size_t n = (size_t)c->W * c->H;
  for (int v = 0; v < 4; v++) {
    c->A[v] = malloc(n * sizeof(double));
    c->B[v] = malloc(n * sizeof(double));
    c->C[v] = malloc(n * sizeof(double));
    c->q[v] = malloc(n * sizeof(double));
    if (v == 0) c->T = malloc(n * sizeof(double));
    c->fx[v] = calloc(n, sizeof(double));
    c->fy[v] = calloc(n, sizeof(double));
    c->Wn[v] = malloc(n * sizeof(double));
    c->Wm[v] = malloc(n * sizeof(double));
    for (size_t m = 0; m < n; m++) c->A[v][m] = c->B[v][m] = c->C[v][m] = c->Wn[v][m] = c->Wm[v][m] = c->Uinf[v];
  }
  c->tag = calloc((size_t)p->nx * p->ny, 1);
  c->precond = p->time_scheme == ORC_TIME_DUAL;
  for (int k = 0; k < 4; k++) c->list[k] = calloc(1, sizeof(orc_stencil));
  return c;
}

void orc_destroy(orc_case *c) {
  if (!c) return;
  for (int v = 0; v < 4; v++) {
    if (v == 0) free(c->T);
    free(c->A[v]); free(c->B[v]); free(c->C[v]); free(c->q[v]); free(c->fx[v]); free(c->fy[v]);
    free(c->Wn[v]); free(c->Wm[v]);
  }
  for (int k = 0; k < 4; k++) free(c->list[k]);
  free(c->tag); free(c->vref); free(c->vx); free(c->vy); free(c->snx); free(c->sny); free(c->vnx); free(c->vny); free(c->vk);
  free(c->snx0); free(c->sny0); free(c->vnx0); free(c->vny0);
  free(c);
}

void orc_get_state(const orc_case *c, double *dst) {
  int nx = c->p.nx, ny = c->p.ny;
  for (int v = 0; v < 4; v++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) dst[((size_t)v * ny + j) * nx + i] = c->A[v][fidx(c, i, j)];
}

void orc_set_state(orc_case *c, const double *src) {
  int nx = c->p.nx, ny = c->p.ny;
  for (int v = 0; v < 4; v++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) c->A[v][fidx(c, i, j)] = src[((size_t)v * ny + j) * nx + i];
}

/* tests: move the case to time t (the next classification poses the body there) */
void orc_set_time(orc_case *c, double t) {
  c->t = t;
  c->classified = 0;
}

void orc_get_tags(const orc_case *c, uint8_t *dst) { memcpy(dst, c->tag, (size_t)c->p.nx * c->p.ny); }
int orc_list_len(const orc_case *c, int kind) { return c->nlist[kind]; }
void orc_get_list(const orc_case *c, int kind, orc_stencil *dst) {
  memcpy(dst, c->list[kind], sizeof(orc_stencil) * c->nlist[kind]);
}
double orc_time(const orc_case *c) { return c->t; }
double orc_last_dt(const orc_case *c) { return c->last_dt; }
