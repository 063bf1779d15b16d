/*
 * FP64 CPU oracle of the 3-D flow solver -- TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The method of arXiv 1912.11908 on one uniform 3-D block around a static closed triangulated body:
 *   Sec. 2      WENO5 on (rho, u, v, w, p), low-diffusion flux splitting LDFSS(0), second-order central
 *               viscous flux, explicit SSP-RK3 stages (the 2-D oracle's readings)
 *   Sec. 3.2    ray-casting classification and tagging (orc_classify_points_3d, orc_tags_3d in oracle.c)
 *   Sec. 4.1-2  closest feature and pseudo-normal (orc_closest_3d in oracle.c)
 *   Sec. 4.3-6  reconstruction of IB nodes along the local normal; Sec. 5 three ghost layers
 *   Sec. 6      surface force (Eq. 9)
 * Every face flux, the stage update and the halo fill are the 2-D oracle's with the third direction added
 * term by term in the same order, so that a field constant along one axis evolves exactly as the 2-D oracle
 * evolves it in the other two (the pin of this file).
 *
 * Readings (3-D only; the 2-D readings of oracle.c carry over):
 *   - boundary point: P' of a listed node X is the foot of X on the plane through its closest surface point
 *     C normal to the local normal n, P' = X - xi_node n with xi_node = (X - C).n.  On a face P' = C; at an
 *     edge or a vertex P' is C moved within that tangent plane (O(h^2) off a smooth surface);
 *   - probes: an IB node's probe lies one cell diagonal h = sqrt(dx^2 + dy^2 + dz^2) beyond the node along
 *     n; a ghost node's image point is its mirror image through P' (at least min(dx, dy, dz) / 2 from P');
 *     either is pushed out by min(dx, dy, dz), up to three times, while its cube has no valid corner;
 *   - interpolation (Sec. 4.6 in 3-D): over the cube of the eight cell centres around the point, trilinear
 *     when all eight are valid, else inverse-distance weights 1 / r^2 over the valid ones (a corner hit
 *     exactly takes all the weight); IB probes use fluid corners, ghost image points fluid and IB corners;
 *   - static wall: zero velocity at P' (Eq. 4, linear along n through the probe), zero normal gradient of
 *     pressure (Eq. 5-6 with no wall acceleration) and of temperature (Eq. 8);
 *   - forces: midpoint rule per triangle, the probe one cell diagonal out along the face normal from the
 *     triangle's centroid, wall pressure the probe's, wall shear mu (u_P - (u_P.n) n) / xi.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NG3 3 /* halo / ghost layers of the five-point WENO stencil (Sec. 5) */

struct orc3_case {
  orc3_params p;
  double *verts;
  int *tris;
  int W, H, D;
  long ncell;
  double dx, dy, dz, h, dmin;
  double R, cp, mu, kappa, pinf;
  double Uinf[5];
  double *A[5], *B[5], *C[5];
  double *q[5]; /* rho, u, v, w, p over the full array */
  double *T;
  double *f[3][5]; /* face fluxes: face i + 1/2 (j + 1/2, k + 1/2) stored at the lower cell */
  uint8_t *tag;
  int nlist[4];
  orc3_stencil *list[4];
  double t, last_dt;
  int classified, nerr;
};

static inline long cidx(const orc3_case *c, int i, int j, int k) {
  return ((long)(k + NG3) * c->H + (j + NG3)) * c->W + (i + NG3);
}

/* primitives (p, u, v, w, T) of a conserved state (Sec. 4.4) and back */
static inline void cons_to_prim3(const orc3_case *c, double *const U[5], long m, double q[5]) {
  double g = c->p.gamma, r = U[0][m];
  double u = U[1][m] / r, v = U[2][m] / r, w = U[3][m] / r;
  double pr = (g - 1.0) * (U[4][m] - 0.5 * r * (u * u + v * v + w * w));
  q[0] = pr;
  q[1] = u;
  q[2] = v;
  q[3] = w;
  q[4] = pr / (r * c->R);
}

static inline void prim_to_cons3(const orc3_case *c, const double q[5], double U[5]) {
  double g = c->p.gamma;
  double r = q[0] / (c->R * q[4]);
  U[0] = r;
  U[1] = r * q[1];
  U[2] = r * q[2];
  U[3] = r * q[3];
  U[4] = q[0] / (g - 1.0) + 0.5 * r * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
}

/* ------------------------------------------------------------------------- */
/* Sec. 4.6 in 3-D: interpolation cube and weights around X.                 */
/* ------------------------------------------------------------------------- */
#define A3_FLUID (1u << ORC_FLUID)
#define A3_FLUID_IB ((1u << ORC_FLUID) | (1u << ORC_IB))

static int interp_cube(const orc3_case *c, const double X[3], unsigned allowed, int32_t o[3], double w[8]) {
  const orc3_params *p = &c->p;
  const double d[3] = {c->dx, c->dy, c->dz};
  const int n[3] = {p->nx, p->ny, p->nz};
  for (int a = 0; a < 3; a++) o[a] = (int32_t)floor((X[a] - p->lo[a]) / d[a] - 0.5);
  int mask = 0;
  for (int b = 0; b < 8; b++) {
    int ci = o[0] + (b & 1), cj = o[1] + (b >> 1 & 1), ck = o[2] + (b >> 2);
    w[b] = 0.0;
    if (ci < 0 || ci >= n[0] || cj < 0 || cj >= n[1] || ck < 0 || ck >= n[2]) continue;
    if (allowed & (1u << c->tag[((long)ck * n[1] + cj) * n[0] + ci])) mask |= 1 << b;
  }
  if (mask == 255) {
    double f[3];
    for (int a = 0; a < 3; a++) {
      double c0 = p->lo[a] + ((double)o[a] + 0.5) * d[a];
      f[a] = (X[a] - c0) / d[a];
    }
    for (int b = 0; b < 8; b++) {
      double wx = (b & 1) ? f[0] : 1.0 - f[0];
      double wy = (b >> 1 & 1) ? f[1] : 1.0 - f[1];
      double wz = (b >> 2) ? f[2] : 1.0 - f[2];
      w[b] = wx * wy * wz;
    }
  } else if (mask != 0) {
    double inv[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int hit = -1;
    for (int b = 0; b < 8 && hit < 0; b++) {
      if (!(mask >> b & 1)) continue;
      double r2 = 0.0;
      for (int a = 0; a < 3; a++) {
        int idx = o[a] + (a == 0 ? (b & 1) : a == 1 ? (b >> 1 & 1) : (b >> 2));
        double xc = p->lo[a] + ((double)idx + 0.5) * d[a];
        double r = X[a] - xc;
        r2 = r2 + r * r;
      }
      if (r2 == 0.0) hit = b;
      else inv[b] = 1.0 / r2;
    }
    if (hit >= 0) {
      w[hit] = 1.0;
    } else {
      double s = 0.0;
      for (int b = 0; b < 8; b++)
        if (mask >> b & 1) s += inv[b];
      for (int b = 0; b < 8; b++)
        if (mask >> b & 1) w[b] = inv[b] / s;
    }
  }
  return mask;
}

/* ------------------------------------------------------------------------- */
/* Sec. 4.3 + Sec. 5: one stencil per listed node from its closest point C,  */
/* local normal n and feature kind.                                          */
/* ------------------------------------------------------------------------- */
static void build_stencil3(orc3_case *c, int node, int kind, const double C[3], const double n[3], int region,
                           orc3_stencil *s) {
  const orc3_params *p = &c->p;
  const double d[3] = {c->dx, c->dy, c->dz};
  int ijk[3] = {node % p->nx, (node / p->nx) % p->ny, node / (p->nx * p->ny)};
  double X[3];
  for (int a = 0; a < 3; a++) X[a] = p->lo[a] + ((double)ijk[a] + 0.5) * d[a];
  double xi_node = (X[0] - C[0]) * n[0] + (X[1] - C[1]) * n[1] + (X[2] - C[2]) * n[2];
  double b[3];
  for (int a = 0; a < 3; a++) b[a] = X[a] - xi_node * n[a];
  double xi_probe;
  if (kind == 0) {
    xi_probe = xi_node + c->h; /* one cell diagonal beyond the IB node */
  } else {
    xi_probe = -xi_node;       /* mirror image point (Sec. 5) */
    if (xi_probe < 0.5 * c->dmin) xi_probe = 0.5 * c->dmin;
  }
  unsigned allowed = kind == 0 ? A3_FLUID : A3_FLUID_IB;
  int32_t o[3] = {0, 0, 0};
  int mask = 0, nstep = 0;
  for (;;) {
    double P[3];
    for (int a = 0; a < 3; a++) P[a] = b[a] + xi_probe * n[a];
    mask = interp_cube(c, P, allowed, o, s->w);
    if (mask != 0 || nstep == 3) break;
    xi_probe = xi_probe + c->dmin;
    nstep++;
  }
  if (mask == 0) c->nerr++;
  s->node = node;
  s->kind = kind;
  s->region = region;
  s->nstep = nstep;
  s->i0 = o[0];
  s->j0 = o[1];
  s->k0 = o[2];
  s->mask = mask;
  for (int a = 0; a < 3; a++) {
    s->n[a] = n[a];
    s->b[a] = b[a];
  }
  s->xi_node = xi_node;
  s->xi_probe = xi_probe;
}

int orc3_classify(orc3_case *c) {
  const orc3_params *p = &c->p;
  long nn = (long)p->nx * p->ny * p->nz;
  const double d[3] = {c->dx, c->dy, c->dz};
  uint8_t *solid = calloc(nn, 1);
  if (p->ntri > 0) {
    double *pts = malloc(sizeof(double) * 3 * nn);
    for (long m = 0; m < nn; m++) {
      int ijk[3] = {(int)(m % p->nx), (int)((m / p->nx) % p->ny), (int)(m / ((long)p->nx * p->ny))};
      for (int a = 0; a < 3; a++) pts[3 * m + a] = p->lo[a] + ((double)ijk[a] + 0.5) * d[a];
    }
    orc_classify_points_3d(p->nv, c->verts, p->ntri, c->tris, (int)nn, pts, solid);
    free(pts);
  }
  orc_tags_3d(p->nx, p->ny, p->nz, solid, c->tag);
  free(solid);
  c->nerr = 0;
  for (int kind = 0; kind < 4; kind++) {
    uint8_t want = (uint8_t)(kind == 0 ? ORC_IB : ORC_G1 + kind - 1);
    int n = 0;
    for (long m = 0; m < nn; m++) n += c->tag[m] == want;
    free(c->list[kind]);
    c->list[kind] = calloc(n > 0 ? n : 1, sizeof(orc3_stencil));
    c->nlist[kind] = n;
    if (!n) continue;
    int *nodes = malloc(sizeof(int) * n);
    double *pts = malloc(sizeof(double) * 3 * n), *cpt = malloc(sizeof(double) * 3 * n),
           *nrm = malloc(sizeof(double) * 3 * n);
    int32_t *fk = malloc(sizeof(int32_t) * n);
    int w = 0;
    for (long m = 0; m < nn; m++)
      if (c->tag[m] == want) {
        int ijk[3] = {(int)(m % p->nx), (int)((m / p->nx) % p->ny), (int)(m / ((long)p->nx * p->ny))};
        for (int a = 0; a < 3; a++) pts[3 * w + a] = p->lo[a] + ((double)ijk[a] + 0.5) * d[a];
        nodes[w++] = (int)m;
      }
    orc_closest_3d(p->nv, c->verts, p->ntri, c->tris, n, pts, cpt, nrm, fk);
    for (int e = 0; e < n; e++) build_stencil3(c, nodes[e], kind, cpt + 3 * e, nrm + 3 * e, fk[e], &c->list[kind][e]);
    free(nodes);
    free(pts);
    free(cpt);
    free(nrm);
    free(fk);
  }
  c->classified = 1;
  return c->nerr;
}

/* ------------------------------------------------------------------------- */
/* Sec. 4.4-4.6, Sec. 5: IB nodes from their probes (fluid corners), then    */
/* the three ghost layers from their image points (fluid and IB corners).   */
/* Static wall: u = u_probe xi_node / xi_probe (zero at P', Eq. 4), p and T  */
/* the probe's (zero normal gradient, Eq. 5-6 and 8).                        */
/* ------------------------------------------------------------------------- */
static void reconstruct_set3(orc3_case *c, double *const U[5], const orc3_stencil *s, int n) {
  const orc3_params *p = &c->p;
  for (int e = 0; e < n; e++) {
    const orc3_stencil *st = &s[e];
    if (st->mask == 0) continue;
    double qp[5] = {0, 0, 0, 0, 0};
    for (int b = 0; b < 8; b++) {
      if (!(st->mask >> b & 1)) continue;
      long id = cidx(c, st->i0 + (b & 1), st->j0 + (b >> 1 & 1), st->k0 + (b >> 2));
      double qk[5];
      cons_to_prim3(c, U, id, qk);
      for (int v = 0; v < 5; v++) qp[v] += st->w[b] * qk[v];
    }
    double ratio = st->xi_node / st->xi_probe;
    double q[5] = {qp[0], qp[1] * ratio, qp[2] * ratio, qp[3] * ratio, qp[4]};
    double Un[5];
    prim_to_cons3(c, q, Un);
    int i = st->node % p->nx, j = (st->node / p->nx) % p->ny, k = st->node / (p->nx * p->ny);
    long id = cidx(c, i, j, k);
    for (int v = 0; v < 5; v++) U[v][id] = Un[v];
  }
}

static void reconstruct3(orc3_case *c, double *const U[5]) {
  for (int k = 0; k < 4; k++) reconstruct_set3(c, U, c->list[k], c->nlist[k]);
}

void orc3_reconstruct(orc3_case *c) {
  if (!c->classified) orc3_classify(c);
  reconstruct3(c, c->A);
}

/* ------------------------------------------------------------------------- */
/* Domain halos: free-stream Dirichlet, zero-gradient outflow, or periodic.  */
/* z sides over the interior (i, j), then y sides over interior i and every */
/* k, then x sides over every (j, k).                                        */
/* ------------------------------------------------------------------------- */
static void domain_bc3(orc3_case *c, double *const U[5]) {
  const orc3_params *p = &c->p;
  int nx = p->nx, ny = p->ny, nz = p->nz;
  for (int side = 4; side < 6; side++)
    for (int g = 1; g <= NG3; g++)
      for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
          int k = side == 4 ? -g : nz - 1 + g;
          long src;
          if (p->bc[side] == ORC_BC_PERIODIC) src = cidx(c, i, j, side == 4 ? nz - g : g - 1);
          else if (p->bc[side] == ORC_BC_OUTFLOW) src = cidx(c, i, j, side == 4 ? 0 : nz - 1);
          else src = -1;
          long dst = cidx(c, i, j, k);
          for (int v = 0; v < 5; v++) U[v][dst] = src < 0 ? c->Uinf[v] : U[v][src];
        }
  for (int side = 2; side < 4; side++)
    for (int g = 1; g <= NG3; g++)
      for (int k = -NG3; k < nz + NG3; k++)
        for (int i = 0; i < nx; i++) {
          int j = side == 2 ? -g : ny - 1 + g;
          long src;
          if (p->bc[side] == ORC_BC_PERIODIC) src = cidx(c, i, side == 2 ? ny - g : g - 1, k);
          else if (p->bc[side] == ORC_BC_OUTFLOW) src = cidx(c, i, side == 2 ? 0 : ny - 1, k);
          else src = -1;
          long dst = cidx(c, i, j, k);
          for (int v = 0; v < 5; v++) U[v][dst] = src < 0 ? c->Uinf[v] : U[v][src];
        }
  for (int side = 0; side < 2; side++)
    for (int g = 1; g <= NG3; g++)
      for (int k = -NG3; k < nz + NG3; k++)
        for (int j = -NG3; j < ny + NG3; j++) {
          int i = side == 0 ? -g : nx - 1 + g;
          long src;
          if (p->bc[side] == ORC_BC_PERIODIC) src = cidx(c, side == 0 ? nx - g : g - 1, j, k);
          else if (p->bc[side] == ORC_BC_OUTFLOW) src = cidx(c, side == 0 ? 0 : nx - 1, j, k);
          else src = -1;
          long dst = cidx(c, i, j, k);
          for (int v = 0; v < 5; v++) U[v][dst] = src < 0 ? c->Uinf[v] : U[v][src];
        }
}

/* ------------------------------------------------------------------------- */
/* Sec. 2: fifth-order WENO states of (rho, u, v, w, p) at the face between  */
/* cells s[2] and s[3] of a six-cell strip (orc_weno5), first order where a  */
/* reconstructed density or pressure is not positive.                        */
/* ------------------------------------------------------------------------- */
static void face_states3(const double s[6][5], double qL[5], double qR[5]) {
  for (int v = 0; v < 5; v++) {
    double fl[5] = {s[0][v], s[1][v], s[2][v], s[3][v], s[4][v]};
    double fr[5] = {s[5][v], s[4][v], s[3][v], s[2][v], s[1][v]};
    qL[v] = orc_weno5(fl);
    qR[v] = orc_weno5(fr);
  }
  if (!(qL[0] > 0.0) || !(qL[4] > 0.0) || !(qR[0] > 0.0) || !(qR[4] > 0.0)) {
    for (int v = 0; v < 5; v++) {
      qL[v] = s[2][v];
      qR[v] = s[3][v];
    }
  }
}

/* ------------------------------------------------------------------------- */
/* Sec. 2: LDFSS(0) across a face of unit normal (nxf, nyf, nzf); the 2-D    */
/* oracle's reading (plain LDFSS, Mr^2 = 1, for explicit time stepping)      */
/* with the third velocity component carried like the others.               */
/* ------------------------------------------------------------------------- */
static void ldfss3(const double qL[5], const double qR[5], double nxf, double nyf, double nzf, double gamma,
                   double F[5]) {
  const double mr2 = 1.0;
  double rL = qL[0], uL = qL[1], vL = qL[2], wL = qL[3], pL = qL[4];
  double rR = qR[0], uR = qR[1], vR = qR[2], wR = qR[3], pR = qR[4];
  double cL = sqrt(gamma * pL / rL), cR = sqrt(gamma * pR / rR);
  double HL = gamma / (gamma - 1.0) * pL / rL + 0.5 * (uL * uL + vL * vL + wL * wL);
  double HR = gamma / (gamma - 1.0) * pR / rR + 0.5 * (uR * uR + vR * vR + wR * wR);
  double unL = uL * nxf + vL * nyf + wL * nzf, unR = uR * nxf + vR * nyf + wR * nzf;
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
  double PpL = 0.25 * (ML + 1.0) * (ML + 1.0) * (2.0 - ML);
  double PmR = 0.25 * (MR - 1.0) * (MR - 1.0) * (2.0 + MR);
  double DL = aL * (1.0 + bL) - bL * PpL;
  double DR = aR * (1.0 + bR) - bR * PmR;
  double mL = rL * cs * Cp, mR = rR * cs * Cm;
  double ph = DL * pL + DR * pR;
  F[0] = mL + mR;
  F[1] = mL * uL + mR * uR + ph * nxf;
  F[2] = mL * vL + mR * vR + ph * nyf;
  F[3] = mL * wL + mR * wR + ph * nzf;
  F[4] = mL * HL + mR * HR;
}

/* ------------------------------------------------------------------------- */
/* Sec. 2: face fluxes, inviscid (WENO5 + LDFSS) minus viscous (second-order */
/* central: normal derivatives across the face, tangential ones from the     */
/* four-cell average of central differences; Stokes hypothesis).             */
/* ------------------------------------------------------------------------- */
static void residual3(orc3_case *c, double *const U[5]) {
  const orc3_params *p = &c->p;
  int nx = p->nx, ny = p->ny, nz = p->nz;
  double g = p->gamma, R = c->R, mu = c->mu, kap = c->kappa;
  double *const *Q = c->q;
  for (long m = 0; m < c->ncell; m++) {
    double r = U[0][m], u = U[1][m] / r, v = U[2][m] / r, w = U[3][m] / r;
    double pr = (g - 1.0) * (U[4][m] - 0.5 * r * (u * u + v * v + w * w));
    Q[0][m] = r;
    Q[1][m] = u;
    Q[2][m] = v;
    Q[3][m] = w;
    Q[4][m] = pr;
    c->T[m] = pr / (r * R);
  }
  const double *Tm = c->T;
  /* x-faces i + 1/2, i in [-1, nx - 1] */
#pragma omp parallel for schedule(static) collapse(2)
  for (int k = 0; k < nz; k++)
    for (int j = 0; j < ny; j++)
      for (int i = -1; i < nx; i++) {
        double s[6][5];
        for (int t = 0; t < 6; t++)
          for (int v = 0; v < 5; v++) s[t][v] = Q[v][cidx(c, i - 2 + t, j, k)];
        double qL[5], qR[5], F[5];
        face_states3(s, qL, qR);
        ldfss3(qL, qR, 1.0, 0.0, 0.0, g, F);
        long a = cidx(c, i, j, k), b = cidx(c, i + 1, j, k);
        long an = cidx(c, i, j + 1, k), as = cidx(c, i, j - 1, k), bn = cidx(c, i + 1, j + 1, k),
             bs = cidx(c, i + 1, j - 1, k);
        long at = cidx(c, i, j, k + 1), ab = cidx(c, i, j, k - 1), bt = cidx(c, i + 1, j, k + 1),
             bb = cidx(c, i + 1, j, k - 1);
        double ux = (Q[1][b] - Q[1][a]) / c->dx, vx = (Q[2][b] - Q[2][a]) / c->dx;
        double wx = (Q[3][b] - Q[3][a]) / c->dx, Tx = (Tm[b] - Tm[a]) / c->dx;
        double uy = (Q[1][an] - Q[1][as] + Q[1][bn] - Q[1][bs]) / (4.0 * c->dy);
        double vy = (Q[2][an] - Q[2][as] + Q[2][bn] - Q[2][bs]) / (4.0 * c->dy);
        double uz = (Q[1][at] - Q[1][ab] + Q[1][bt] - Q[1][bb]) / (4.0 * c->dz);
        double wz = (Q[3][at] - Q[3][ab] + Q[3][bt] - Q[3][bb]) / (4.0 * c->dz);
        double txx = mu * ((4.0 / 3.0) * ux - (2.0 / 3.0) * (vy + wz));
        double txy = mu * (uy + vx);
        double txz = mu * (uz + wx);
        double qx = -kap * Tx;
        double uf = 0.5 * (Q[1][a] + Q[1][b]), vf = 0.5 * (Q[2][a] + Q[2][b]), wf = 0.5 * (Q[3][a] + Q[3][b]);
        c->f[0][0][a] = F[0];
        c->f[0][1][a] = F[1] - txx;
        c->f[0][2][a] = F[2] - txy;
        c->f[0][3][a] = F[3] - txz;
        c->f[0][4][a] = F[4] - (uf * txx + vf * txy + wf * txz - qx);
      }
  /* y-faces j + 1/2, j in [-1, ny - 1] */
#pragma omp parallel for schedule(static) collapse(2)
  for (int k = 0; k < nz; k++)
    for (int j = -1; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        double s[6][5];
        for (int t = 0; t < 6; t++)
          for (int v = 0; v < 5; v++) s[t][v] = Q[v][cidx(c, i, j - 2 + t, k)];
        double qL[5], qR[5], F[5];
        face_states3(s, qL, qR);
        ldfss3(qL, qR, 0.0, 1.0, 0.0, g, F);
        long a = cidx(c, i, j, k), b = cidx(c, i, j + 1, k);
        long ae = cidx(c, i + 1, j, k), aw = cidx(c, i - 1, j, k), be = cidx(c, i + 1, j + 1, k),
             bw = cidx(c, i - 1, j + 1, k);
        long at = cidx(c, i, j, k + 1), ab = cidx(c, i, j, k - 1), bt = cidx(c, i, j + 1, k + 1),
             bb = cidx(c, i, j + 1, k - 1);
        double uy = (Q[1][b] - Q[1][a]) / c->dy, vy = (Q[2][b] - Q[2][a]) / c->dy;
        double wy = (Q[3][b] - Q[3][a]) / c->dy, Ty = (Tm[b] - Tm[a]) / c->dy;
        double ux = (Q[1][ae] - Q[1][aw] + Q[1][be] - Q[1][bw]) / (4.0 * c->dx);
        double vx = (Q[2][ae] - Q[2][aw] + Q[2][be] - Q[2][bw]) / (4.0 * c->dx);
        double vz = (Q[2][at] - Q[2][ab] + Q[2][bt] - Q[2][bb]) / (4.0 * c->dz);
        double wz = (Q[3][at] - Q[3][ab] + Q[3][bt] - Q[3][bb]) / (4.0 * c->dz);
        double tyy = mu * ((4.0 / 3.0) * vy - (2.0 / 3.0) * (ux + wz));
        double txy = mu * (uy + vx);
        double tyz = mu * (vz + wy);
        double qy = -kap * Ty;
        double uf = 0.5 * (Q[1][a] + Q[1][b]), vf = 0.5 * (Q[2][a] + Q[2][b]), wf = 0.5 * (Q[3][a] + Q[3][b]);
        c->f[1][0][a] = F[0];
        c->f[1][1][a] = F[1] - txy;
        c->f[1][2][a] = F[2] - tyy;
        c->f[1][3][a] = F[3] - tyz;
        c->f[1][4][a] = F[4] - (uf * txy + vf * tyy + wf * tyz - qy);
      }
  /* z-faces k + 1/2, k in [-1, nz - 1] */
#pragma omp parallel for schedule(static) collapse(2)
  for (int k = -1; k < nz; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        double s[6][5];
        for (int t = 0; t < 6; t++)
          for (int v = 0; v < 5; v++) s[t][v] = Q[v][cidx(c, i, j, k - 2 + t)];
        double qL[5], qR[5], F[5];
        face_states3(s, qL, qR);
        ldfss3(qL, qR, 0.0, 0.0, 1.0, g, F);
        long a = cidx(c, i, j, k), b = cidx(c, i, j, k + 1);
        long ae = cidx(c, i + 1, j, k), aw = cidx(c, i - 1, j, k), be = cidx(c, i + 1, j, k + 1),
             bw = cidx(c, i - 1, j, k + 1);
        long an = cidx(c, i, j + 1, k), as = cidx(c, i, j - 1, k), bn = cidx(c, i, j + 1, k + 1),
             bs = cidx(c, i, j - 1, k + 1);
        double uz = (Q[1][b] - Q[1][a]) / c->dz, vz = (Q[2][b] - Q[2][a]) / c->dz;
        double wz = (Q[3][b] - Q[3][a]) / c->dz, Tz = (Tm[b] - Tm[a]) / c->dz;
        double ux = (Q[1][ae] - Q[1][aw] + Q[1][be] - Q[1][bw]) / (4.0 * c->dx);
        double wx = (Q[3][ae] - Q[3][aw] + Q[3][be] - Q[3][bw]) / (4.0 * c->dx);
        double vy = (Q[2][an] - Q[2][as] + Q[2][bn] - Q[2][bs]) / (4.0 * c->dy);
        double wy = (Q[3][an] - Q[3][as] + Q[3][bn] - Q[3][bs]) / (4.0 * c->dy);
        double tzz = mu * ((4.0 / 3.0) * wz - (2.0 / 3.0) * (ux + vy));
        double txz = mu * (uz + wx);
        double tyz = mu * (vz + wy);
        double qz = -kap * Tz;
        double uf = 0.5 * (Q[1][a] + Q[1][b]), vf = 0.5 * (Q[2][a] + Q[2][b]), wf = 0.5 * (Q[3][a] + Q[3][b]);
        c->f[2][0][a] = F[0];
        c->f[2][1][a] = F[1] - txz;
        c->f[2][2][a] = F[2] - tyz;
        c->f[2][3][a] = F[3] - tzz;
        c->f[2][4][a] = F[4] - (uf * txz + vf * tyz + wf * tzz - qz);
      }
}

/* SSP-RK3 (Shu-Osher) stage on fluid cells (the 2-D oracle's stage_update). */
static void stage_update3(orc3_case *c, int stage, double *const Un[5], double *const In[5], double *const Out[5],
                          double dt) {
  const orc3_params *p = &c->p;
  int nx = p->nx, ny = p->ny, nz = p->nz;
#pragma omp parallel for schedule(static) collapse(2)
  for (int k = 0; k < nz; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        if (c->tag[((long)k * ny + j) * nx + i] != ORC_FLUID) continue;
        long m = cidx(c, i, j, k), mw = cidx(c, i - 1, j, k), ms = cidx(c, i, j - 1, k), mb = cidx(c, i, j, k - 1);
        for (int v = 0; v < 5; v++) {
          double L = -((c->f[0][v][m] - c->f[0][v][mw]) / c->dx + (c->f[1][v][m] - c->f[1][v][ms]) / c->dy +
                       (c->f[2][v][m] - c->f[2][v][mb]) / c->dz);
          double o;
          if (stage == 1) o = Un[v][m] + dt * L;
          else if (stage == 2) o = 0.75 * Un[v][m] + 0.25 * (In[v][m] + dt * L);
          else o = (1.0 / 3.0) * Un[v][m] + (2.0 / 3.0) * (In[v][m] + dt * L);
          Out[v][m] = o;
        }
      }
}

/* CFL rule over fluid cells:
 * dt = CFL / max[(|u|+c)/dx + (|v|+c)/dy + (|w|+c)/dz + 2 gamma mu/(Pr rho) (1/dx^2 + 1/dy^2 + 1/dz^2)]. */
static double compute_dt3(orc3_case *c) {
  const orc3_params *p = &c->p;
  if (p->dt_fixed > 0.0) return p->dt_fixed;
  double lmax = 0.0, g = p->gamma;
  for (int k = 0; k < p->nz; k++)
    for (int j = 0; j < p->ny; j++)
      for (int i = 0; i < p->nx; i++) {
        if (c->tag[((long)k * p->ny + j) * p->nx + i] != ORC_FLUID) continue;
        long m = cidx(c, i, j, k);
        double q[5];
        cons_to_prim3(c, c->A, m, q);
        double cs = sqrt(g * c->R * q[4]);
        double rho = c->A[0][m];
        double lam = (fabs(q[1]) + cs) / c->dx + (fabs(q[2]) + cs) / c->dy + (fabs(q[3]) + cs) / c->dz +
                     (2.0 * g * c->mu / (p->prandtl * rho)) *
                         (1.0 / (c->dx * c->dx) + 1.0 / (c->dy * c->dy) + 1.0 / (c->dz * c->dz));
        if (lam > lmax) lmax = lam;
      }
  return p->cfl / lmax;
}

int orc3_step(orc3_case *c, int nsteps) {
  for (int s = 0; s < nsteps; s++) {
    if (!c->classified) orc3_classify(c);
    double dt = compute_dt3(c);
    double *const *in[3] = {c->A, c->B, c->C};
    double *const *out[3] = {c->B, c->C, c->A};
    for (int k = 0; k < 3; k++) {
      reconstruct3(c, in[k]);
      domain_bc3(c, in[k]);
      residual3(c, in[k]);
      stage_update3(c, k + 1, c->A, in[k], out[k], dt);
    }
    c->t = c->t + dt;
    c->last_dt = dt;
  }
  return c->nerr;
}

/* ------------------------------------------------------------------------- */
/* Sec. 6, Eq. 9 in 3-D: F = sum over triangles of (-(p_s - p_inf) n +      */
/* tau_w) A at the centroid; p_s and the velocity from the probe one cell    */
/* diagonal out along the face normal (pushed out like a stencil probe),    */
/* tau_w = mu (u_P - (u_P.n) n) / xi for the wall at rest.  Compensated      */
/* (Kahan) sums; C = F / (rho_inf U_ref^2 A_ref / 2).                       */
/* ------------------------------------------------------------------------- */
void orc3_forces(orc3_case *c, double out[6]) {
  const orc3_params *p = &c->p;
  if (!c->classified) orc3_classify(c);
  double S[3] = {0, 0, 0}, K[3] = {0, 0, 0};
  for (int f = 0; f < p->ntri; f++) {
    const double *A = c->verts + 3 * c->tris[3 * f], *B = c->verts + 3 * c->tris[3 * f + 1],
                 *C = c->verts + 3 * c->tris[3 * f + 2];
    double e1[3], e2[3], cr[3], m[3];
    for (int a = 0; a < 3; a++) {
      e1[a] = B[a] - A[a];
      e2[a] = C[a] - A[a];
      m[a] = (A[a] + B[a] + C[a]) / 3.0;
    }
    cr[0] = e1[1] * e2[2] - e1[2] * e2[1];
    cr[1] = e1[2] * e2[0] - e1[0] * e2[2];
    cr[2] = e1[0] * e2[1] - e1[1] * e2[0];
    double len = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
    double n[3] = {cr[0] / len, cr[1] / len, cr[2] / len};
    double area = 0.5 * len;
    double xi = c->h, w[8];
    int32_t o[3];
    int mask = 0;
    for (int st = 0; st <= 3; st++) {
      double P[3] = {m[0] + xi * n[0], m[1] + xi * n[1], m[2] + xi * n[2]};
      mask = interp_cube(c, P, A3_FLUID, o, w);
      if (mask) break;
      if (st < 3) xi = xi + c->dmin;
    }
    if (!mask) continue;
    double qp[5] = {0, 0, 0, 0, 0};
    for (int b = 0; b < 8; b++) {
      if (!(mask >> b & 1)) continue;
      long id = cidx(c, o[0] + (b & 1), o[1] + (b >> 1 & 1), o[2] + (b >> 2));
      double qk[5];
      cons_to_prim3(c, c->A, id, qk);
      for (int v = 0; v < 5; v++) qp[v] += w[b] * qk[v];
    }
    double un = qp[1] * n[0] + qp[2] * n[1] + qp[3] * n[2];
    for (int a = 0; a < 3; a++) {
      double tau = c->mu * (qp[1 + a] - un * n[a]) / xi;
      double fa = (-(qp[0] - c->pinf) * n[a] + tau) * area;
      double y = fa - K[a], t = S[a] + y;
      K[a] = (t - S[a]) - y;
      S[a] = t;
    }
  }
  double qref = 0.5 * p->ref_area;
  for (int a = 0; a < 3; a++) {
    out[a] = S[a] / qref;
    out[3 + a] = S[a];
  }
}

/* ------------------------------------------------------------------------- */
/* setup: free stream rho = 1, T = 1, p = 1/(gamma M^2), R = p, mu = 1/Re,   */
/* k = mu cp / Pr (the 2-D oracle's non-dimensionalisation)                 */
/* ------------------------------------------------------------------------- */
orc3_case *orc3_create(const orc3_params *pp) {
  orc3_case *c = calloc(1, sizeof(orc3_case));
  c->p = *pp;
  const orc3_params *p = &c->p;
  int nv = p->nv > 0 ? p->nv : 0, nt = p->ntri > 0 ? p->ntri : 0;
  c->verts = calloc(3 * (nv > 0 ? nv : 1), sizeof(double));
  c->tris = calloc(3 * (nt > 0 ? nt : 1), sizeof(int));
  if (nv) memcpy(c->verts, pp->verts, sizeof(double) * 3 * nv);
  if (nt) memcpy(c->tris, pp->tris, sizeof(int) * 3 * nt);
  c->p.verts = c->verts;
  c->p.tris = c->tris;
  c->W = p->nx + 2 * NG3;
  c->H = p->ny + 2 * NG3;
  c->D = p->nz + 2 * NG3;
  c->ncell = (long)c->W * c->H * c->D;
  c->dx = (p->hi[0] - p->lo[0]) / p->nx;
  c->dy = (p->hi[1] - p->lo[1]) / p->ny;
  c->dz = (p->hi[2] - p->lo[2]) / p->nz;
  c->h = sqrt(c->dx * c->dx + c->dy * c->dy + c->dz * c->dz);
  c->dmin = fmin(c->dx, fmin(c->dy, c->dz));
  double g = p->gamma;
  c->pinf = 1.0 / (g * p->mach * p->mach);
  c->R = c->pinf;
  c->cp = g * c->R / (g - 1.0);
  c->mu = p->re > 0.0 ? 1.0 / p->re : 0.0;
  c->kappa = c->mu * c->cp / p->prandtl;
  double u = p->uinf[0], v = p->uinf[1], w = p->uinf[2];
  c->Uinf[0] = 1.0;
  c->Uinf[1] = u;
  c->Uinf[2] = v;
  c->Uinf[3] = w;
  c->Uinf[4] = c->pinf / (g - 1.0) + 0.5 * (u * u + v * v + w * w);
  for (int k = 0; k < 5; k++) {
    c->A[k] = malloc(sizeof(double) * c->ncell);
    c->B[k] = malloc(sizeof(double) * c->ncell);
    c->C[k] = malloc(sizeof(double) * c->ncell);
    c->q[k] = malloc(sizeof(double) * c->ncell);
    for (int d = 0; d < 3; d++) c->f[d][k] = calloc(c->ncell, sizeof(double));
    for (long m = 0; m < c->ncell; m++) c->A[k][m] = c->B[k][m] = c->C[k][m] = c->Uinf[k];
  }
  c->T = malloc(sizeof(double) * c->ncell);
  c->tag = calloc((size_t)p->nx * p->ny * p->nz, 1);
  return c;
}

void orc3_destroy(orc3_case *c) {
  if (!c) return;
  for (int k = 0; k < 5; k++) {
    free(c->A[k]);
    free(c->B[k]);
    free(c->C[k]);
    free(c->q[k]);
    for (int d = 0; d < 3; d++) free(c->f[d][k]);
  }
  for (int k = 0; k < 4; k++) free(c->list[k]);
  free(c->T);
  free(c->tag);
  free(c->verts);
  free(c->tris);
  free(c);
}

void orc3_get_state(const orc3_case *c, double *dst) {
  const orc3_params *p = &c->p;
  long n = 0;
  for (int v = 0; v < 5; v++)
    for (int k = 0; k < p->nz; k++)
      for (int j = 0; j < p->ny; j++)
        for (int i = 0; i < p->nx; i++) dst[n++] = c->A[v][cidx(c, i, j, k)];
}

void orc3_set_state(orc3_case *c, const double *src) {
  const orc3_params *p = &c->p;
  long n = 0;
  for (int v = 0; v < 5; v++)
    for (int k = 0; k < p->nz; k++)
      for (int j = 0; j < p->ny; j++)
        for (int i = 0; i < p->nx; i++) c->A[v][cidx(c, i, j, k)] = src[n++];
}

void orc3_get_tags(const orc3_case *c, uint8_t *dst) {
  memcpy(dst, c->tag, (size_t)c->p.nx * c->p.ny * c->p.nz);
}
int orc3_list_len(const orc3_case *c, int kind) { return c->nlist[kind]; }
void orc3_get_list(const orc3_case *c, int kind, orc3_stencil *dst) {
  memcpy(dst, c->list[kind], sizeof(orc3_stencil) * c->nlist[kind]);
}
double orc3_time(const orc3_case *c) { return c->t; }
double orc3_last_dt(const orc3_case *c) { return c->last_dt; }
