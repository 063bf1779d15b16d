// 3-D flow on the GPU in FP64 (Sec. 2-6 of arXiv 1912.11908 on one uniform 3-D block around a static closed
// triangulated body): explicit SSP-RK3 steps, each stage
//   IB nodes from their probes and the three ghost layers from their image points (Sec. 4.3-4.6, Sec. 5),
//   domain halos, primitives, the face fluxes of the three directions (WENO5 on (rho, u, v, w, p), LDFSS(0),
//   central viscous flux with the Stokes hypothesis; Sec. 2) and the stage update of the fluid cells,
// and Eq. 9's force over the triangles.  Classification, tags, lists and the stencils of the listed nodes and
// of the force probes come from the 3-D pre-processing (geometry3d.cu), once at creation (the body is static).
//
// Layout: structure of arrays over the cells with three halo layers, cell (i, j, k) of the (nx + 6) x (ny + 6)
// x (nz + 6) array at ((k + 3) H + j + 3) W + i + 3; face i + 1/2 (j + 1/2, k + 1/2) of a direction is stored
// at its lower cell.  One thread per cell, per face or per listed node.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "ibm.h"

extern "C" ibm_status ibm__noalloc_fail(ibm_status s, const char *msg);
ibm_status ibm__body3d_stencils(ibm_body3d *b, double h, double dmin, ibm_stencil3d *out, int *nerr,
                                const uint8_t **tags, const int **counts, int *cap);
ibm_status ibm__surface3d_stencils(ibm_body3d *b, const double *mn, int ntri, double h, double dmin,
                                   ibm_stencil3d *out);
int ibm__body3d_capacity(const ibm_body3d *b);

namespace {

constexpr int NG = 3;
constexpr int TB = 256;        // threads per block of the list kernels
constexpr int BX = 32, BY = 4; // block of the per-cell and per-face kernels: 32 cells along x, 4 rows
constexpr int TC = BX * BY;
constexpr uint8_t TAG_FLUID = IBM_TAG_FLUID;

struct Grid3 {
  int nx, ny, nz, W, H, D;
  long long plane, ncell;
  double dx, dy, dz, idx, idy, idz;
  double lo[3];
  int bc[6];
};

struct Phys3 {
  double gamma, R, mu, kappa, prandtl, cfl, pinf, dt_fixed;
  double Uinf[5];
};

struct F5 {
  double *v[5];
};
struct F6 {
  double *v[6];  // rho, u, v, w, p, T
};

__device__ __forceinline__ long long cid(const Grid3 &g, int i, int j, int k) {
  return ((long long)(k + NG) * g.H + (j + NG)) * g.W + (i + NG);
}

// Sec. 2: WENO5 (Jiang-Shu indicators, linear weights 1/10, 6/10, 3/10, eps = 1e-6), left-biased value at the
// face between f[2] and f[3] of f[0..4]
__device__ __forceinline__ double weno5(double f0, double f1, double f2, double f3, double f4) {
  const double eps = 1e-6;
  double a = f0 - 2.0 * f1 + f2, b = f0 - 4.0 * f1 + 3.0 * f2;
  const double b0 = (13.0 / 12.0) * a * a + 0.25 * b * b;
  a = f1 - 2.0 * f2 + f3;
  b = f1 - f3;
  const double b1 = (13.0 / 12.0) * a * a + 0.25 * b * b;
  a = f2 - 2.0 * f3 + f4;
  b = 3.0 * f2 - 4.0 * f3 + f4;
  const double b2 = (13.0 / 12.0) * a * a + 0.25 * b * b;
  const double q0 = (2.0 * f0 - 7.0 * f1 + 11.0 * f2) * (1.0 / 6.0);
  const double q1 = (-f1 + 5.0 * f2 + 2.0 * f3) * (1.0 / 6.0);
  const double q2 = (2.0 * f2 + 5.0 * f3 - f4) * (1.0 / 6.0);
  const double e0 = eps + b0, e1 = eps + b1, e2 = eps + b2;
  // alpha_k = d_k / e_k^2 over a common denominator: one division
  const double s0 = e1 * e1 * e2 * e2, s1 = e0 * e0 * e2 * e2, s2 = e0 * e0 * e1 * e1;
  const double a0 = 0.1 * s0, a1 = 0.6 * s1, a2 = 0.3 * s2;
  return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
}

// Sec. 2: LDFSS(0) across a face of unit normal along axis DIR (plain: Mr = 1, so c' = (c_L + c_R) / 2);
// q = (rho, u, v, w, p)
template <int DIR>
__device__ __forceinline__ void ldfss(const double qL[5], const double qR[5], double gamma, double F[5]) {
  const double rL = qL[0], pL = qL[4], rR = qR[0], pR = qR[4];
  const double irL = 1.0 / rL, irR = 1.0 / rR;
  const double cL = sqrt(gamma * pL * irL), cR = sqrt(gamma * pR * irR);
  const double gg = gamma / (gamma - 1.0);
  const double HL = gg * pL * irL + 0.5 * (qL[1] * qL[1] + qL[2] * qL[2] + qL[3] * qL[3]);
  const double HR = gg * pR * irR + 0.5 * (qR[1] * qR[1] + qR[2] * qR[2] + qR[3] * qR[3]);
  const double unL = qL[1 + DIR], unR = qR[1 + DIR];
  const double cs = 0.5 * (cL + cR), ics = 1.0 / cs;
  const double ML = unL * ics, MR = unR * ics;
  const double aL = ML >= 0.0 ? 1.0 : 0.0, aR = MR >= 0.0 ? 0.0 : 1.0;
  const double tL = 1.0 - floor(fabs(ML)), tR = 1.0 - floor(fabs(MR));
  const double bL = -fmax(tL, 0.0), bR = -fmax(tR, 0.0);
  const double MpL = 0.25 * (ML + 1.0) * (ML + 1.0);
  const double MmR = -0.25 * (MR - 1.0) * (MR - 1.0);
  const double CVL = aL * (1.0 + bL) * ML - bL * MpL;
  const double CVR = aR * (1.0 + bR) * MR - bR * MmR;
  const double sq = sqrt(0.5 * (ML * ML + MR * MR)) - 1.0;
  const double Mh = 0.25 * bL * bR * sq * sq;
  const double dp = pL - pR, adp = fabs(dp), ic2 = 0.5 * ics * ics;
  const double MhP = Mh * (1.0 - (dp + adp) * ic2 * irL);
  const double MhM = Mh * (1.0 - (-dp + adp) * ic2 * irR);
  const double Cp = CVL - MhP, Cm = CVR + MhM;
  const double PpL = 0.25 * (ML + 1.0) * (ML + 1.0) * (2.0 - ML);
  const double PmR = 0.25 * (MR - 1.0) * (MR - 1.0) * (2.0 + MR);
  const double DL = aL * (1.0 + bL) - bL * PpL;
  const double DR = aR * (1.0 + bR) - bR * PmR;
  const double mL = rL * cs * Cp, mR = rR * cs * Cm;
  const double ph = DL * pL + DR * pR;
  F[0] = mL + mR;
  F[1] = mL * qL[1] + mR * qR[1];
  F[2] = mL * qL[2] + mR * qR[2];
  F[3] = mL * qL[3] + mR * qR[3];
  F[1 + DIR] += ph;
  F[4] = mL * HL + mR * HR;
}

// primitives (rho, u, v, w, p) and T of every cell, halos included
__global__ void __launch_bounds__(TC) k3_prim(Grid3 g, Phys3 ph, F5 U, F6 Q) {
  const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y;
  if (x >= g.W || y >= g.H) return;
  const long long m = ((long long)blockIdx.z * g.H + y) * g.W + x;
  const double r = U.v[0][m], ir = 1.0 / r;
  const double u = U.v[1][m] * ir, v = U.v[2][m] * ir, w = U.v[3][m] * ir;
  const double p = (ph.gamma - 1.0) * (U.v[4][m] - 0.5 * r * (u * u + v * v + w * w));
  Q.v[0][m] = r;
  Q.v[1][m] = u;
  Q.v[2][m] = v;
  Q.v[3][m] = w;
  Q.v[4][m] = p;
  Q.v[5][m] = p * ir / ph.R;
}

// face fluxes of direction DIR: inviscid (WENO5 states, first order where a density or pressure is not
// positive; LDFSS) minus viscous (normal derivatives across the face, tangential ones from four-cell central
// averages)
template <int DIR>
__global__ void __launch_bounds__(TC) k3_flux(Grid3 g, Phys3 ph, F6 Q, F5 Fo) {
  // faces i + 1/2 (DIR 0) for i in [-1, nx - 1], likewise along y and z; one thread per face
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= g.nx + (DIR == 0) || j >= g.ny + (DIR == 1)) return;
  if (DIR == 0) i -= 1;
  if (DIR == 1) j -= 1;
  if (DIR == 2) k -= 1;
  const long long st = DIR == 0 ? 1 : DIR == 1 ? (long long)g.W : g.plane;
  const long long a = cid(g, i, j, k), b = a + st;
  double qL[5], qR[5];
  for (int v = 0; v < 5; v++) {
    const double *q = Q.v[v];
    const double f0 = q[a - 2 * st], f1 = q[a - st], f2 = q[a], f3 = q[b], f4 = q[b + st], f5 = q[b + 2 * st];
    qL[v] = weno5(f0, f1, f2, f3, f4);
    qR[v] = weno5(f5, f4, f3, f2, f1);
  }
  if (!(qL[0] > 0.0) || !(qL[4] > 0.0) || !(qR[0] > 0.0) || !(qR[4] > 0.0)) {
    for (int v = 0; v < 5; v++) {
      qL[v] = Q.v[v][a];
      qR[v] = Q.v[v][b];
    }
  }
  double F[5];
  ldfss<DIR>(qL, qR, ph.gamma, F);
  if (ph.mu > 0.0) {
    // the two tangential directions t1 < t2 and their strides and inverse spacings
    const int t1 = DIR == 0 ? 1 : 0, t2 = DIR == 2 ? 1 : 2;
    const long long s1 = t1 == 0 ? 1 : (long long)g.W, s2 = t2 == 1 ? (long long)g.W : g.plane;
    const double ih[3] = {g.idx, g.idy, g.idz};
    const double in = ih[DIR], i1 = 0.25 * ih[t1], i2 = 0.25 * ih[t2];
    const double *T = Q.v[5];
    double dn[3], d1[3], d2[3];  // d(u, v, w)/dn and the tangential derivatives
    for (int c = 0; c < 3; c++) {
      const double *q = Q.v[1 + c];
      dn[c] = (q[b] - q[a]) * in;
      d1[c] = (q[a + s1] - q[a - s1] + q[b + s1] - q[b - s1]) * i1;
      d2[c] = (q[a + s2] - q[a - s2] + q[b + s2] - q[b - s2]) * i2;
    }
    // velocity gradient G[c][e] = d u_c / d x_e
    double G[3][3];
    for (int c = 0; c < 3; c++) {
      G[c][DIR] = dn[c];
      G[c][t1] = d1[c];
      G[c][t2] = d2[c];
    }
    const double div = G[0][0] + G[1][1] + G[2][2];
    double tau[3];  // row DIR of the viscous stress
    for (int c = 0; c < 3; c++) tau[c] = ph.mu * (G[c][DIR] + G[DIR][c]);
    tau[DIR] = ph.mu * (2.0 * G[DIR][DIR] - (2.0 / 3.0) * div);
    const double qn = -ph.kappa * (T[b] - T[a]) * in;
    double work = 0.0;
    for (int c = 0; c < 3; c++) {
      F[1 + c] -= tau[c];
      work += 0.5 * (Q.v[1 + c][a] + Q.v[1 + c][b]) * tau[c];
    }
    F[4] -= work - qn;
  }
  for (int v = 0; v < 5; v++) Fo.v[v][a] = F[v];
}

// SSP-RK3 stage on the fluid cells: out = Un + dt L, 3/4 Un + 1/4 (in + dt L), 1/3 Un + 2/3 (in + dt L)
__global__ void __launch_bounds__(TC) k3_update(Grid3 g, int stage, F5 Fx, F5 Fy, F5 Fz, F5 Un, F5 In, F5 Out,
                                                const uint8_t *__restrict__ tags, const double *__restrict__ dtp) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  if (tags[((long long)k * g.ny + j) * g.nx + i] != TAG_FLUID) return;
  const long long m = cid(g, i, j, k);
  const double dt = *dtp;
  for (int v = 0; v < 5; v++) {
    const double L = -((Fx.v[v][m] - Fx.v[v][m - 1]) * g.idx + (Fy.v[v][m] - Fy.v[v][m - g.W]) * g.idy +
                       (Fz.v[v][m] - Fz.v[v][m - g.plane]) * g.idz);
    double o;
    if (stage == 1) o = Un.v[v][m] + dt * L;
    else if (stage == 2) o = 0.75 * Un.v[v][m] + 0.25 * (In.v[v][m] + dt * L);
    else o = (1.0 / 3.0) * Un.v[v][m] + (2.0 / 3.0) * (In.v[v][m] + dt * L);
    Out.v[v][m] = o;
  }
}

// CFL rule: the largest (|u|+c)/dx + (|v|+c)/dy + (|w|+c)/dz + 2 gamma mu/(Pr rho)(1/dx^2 + 1/dy^2 + 1/dz^2)
// over the fluid cells (max of positive doubles through their bit patterns: order independent)
__global__ void __launch_bounds__(TC) k3_lambda(Grid3 g, Phys3 ph, F5 U, const uint8_t *__restrict__ tags,
                                                unsigned long long *__restrict__ lmax) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  double lam = 0.0;
  if (i < g.nx && j < g.ny && tags[((long long)k * g.ny + j) * g.nx + i] == TAG_FLUID) {
    const long long m = cid(g, i, j, k);
    const double r = U.v[0][m], ir = 1.0 / r;
    const double u = U.v[1][m] * ir, v = U.v[2][m] * ir, w = U.v[3][m] * ir;
    const double p = (ph.gamma - 1.0) * (U.v[4][m] - 0.5 * r * (u * u + v * v + w * w));
    const double c = sqrt(ph.gamma * ph.R * (p * ir / ph.R));
    lam = (fabs(u) + c) * g.idx + (fabs(v) + c) * g.idy + (fabs(w) + c) * g.idz +
          (2.0 * ph.gamma * ph.mu / (ph.prandtl * r)) * (g.idx * g.idx + g.idy * g.idy + g.idz * g.idz);
  }
  for (int o = 16; o > 0; o >>= 1) lam = fmax(lam, __shfl_xor_sync(0xffffffffu, lam, o));
  if ((threadIdx.x & 31) == 0 && lam > 0.0) atomicMax(lmax, (unsigned long long)__double_as_longlong(lam));
}

// domain halos in closed form: the free stream if the cell lies beyond a free-stream side along any axis,
// else the interior cell reached by mapping each out-of-range index (periodic wrap or zero-gradient clamp).
// One thread per halo cell: the two z slabs (every x, y), the two y slabs of the interior z range (every x),
// the two x slabs of the interior y, z range
__global__ void __launch_bounds__(TB) k3_halo(Grid3 g, Phys3 ph, F5 U) {
  const int t = blockIdx.x * TB + threadIdx.x;
  const int nzs = 2 * NG * g.W * g.H, nys = 2 * NG * g.nz * g.W, nxs = 2 * NG * g.nz * g.ny;
  int x, y, z;
  if (t < nzs) {
    const int zz = t / (g.W * g.H), rem = t - zz * (g.W * g.H);
    z = zz < NG ? zz : g.nz + zz;
    y = rem / g.W;
    x = rem - y * g.W;
  } else if (t < nzs + nys) {
    const int u = t - nzs, zz = u / (2 * NG * g.W), rem = u - zz * (2 * NG * g.W), yy = rem / g.W;
    z = NG + zz;
    y = yy < NG ? yy : g.ny + yy;
    x = rem - yy * g.W;
  } else if (t < nzs + nys + nxs) {
    const int u = t - nzs - nys, zz = u / (2 * NG * g.ny), rem = u - zz * (2 * NG * g.ny), yy = rem / (2 * NG);
    const int xx = rem - yy * (2 * NG);
    z = NG + zz;
    y = NG + yy;
    x = xx < NG ? xx : g.nx + xx;
  } else {
    return;
  }
  const long long m = ((long long)z * g.H + y) * g.W + x;
  const int I[3] = {x - NG, y - NG, z - NG};
  const int n[3] = {g.nx, g.ny, g.nz};
  int S[3];
  bool fs = false;
  for (int a = 0; a < 3; a++) {
    S[a] = I[a];
    if (I[a] >= 0 && I[a] < n[a]) continue;
    const int bc = g.bc[2 * a + (I[a] < 0 ? 0 : 1)];
    if (bc == IBM_BC_PERIODIC) S[a] = I[a] < 0 ? I[a] + n[a] : I[a] - n[a];
    else if (bc == IBM_BC_OUTFLOW) S[a] = I[a] < 0 ? 0 : n[a] - 1;
    else fs = true;
  }
  if (fs) {
    for (int v = 0; v < 5; v++) U.v[v][m] = ph.Uinf[v];
  } else {
    const long long src = cid(g, S[0], S[1], S[2]);
    for (int v = 0; v < 5; v++) U.v[v][m] = U.v[v][src];
  }
}

// Sec. 4.4-4.6 and Sec. 5 with a static wall: the node takes the probe's (image point's) pressure and
// temperature and its velocity scaled by xi_node / xi_probe (zero at P').  Eight lanes per node, one cube corner
// each, the weighted sums formed by a fixed shuffle tree (a warp holds four nodes)
__global__ void __launch_bounds__(128) k3_reconstruct(Grid3 g, Phys3 ph, F5 U, const ibm_stencil3d *__restrict__ st,
                                                      int first, int count) {
  const int t = blockIdx.x * 128 + threadIdx.x;
  const int e = t >> 3, b = t & 7;
  const bool live = e < count;
  const ibm_stencil3d *sp = st + first + (live ? e : 0);
  const int mask = live ? sp->mask : 0;
  double q[5] = {0.0, 0.0, 0.0, 0.0, 0.0};  // this corner's weighted p, u, v, w, T
  if (mask >> b & 1) {
    const long long id = cid(g, sp->i0 + (b & 1), sp->j0 + (b >> 1 & 1), sp->k0 + (b >> 2));
    const double r = U.v[0][id], ir = 1.0 / r;
    const double u = U.v[1][id] * ir, v = U.v[2][id] * ir, w = U.v[3][id] * ir;
    const double p = (ph.gamma - 1.0) * (U.v[4][id] - 0.5 * r * (u * u + v * v + w * w));
    const double wb = sp->w[b];
    q[0] = wb * p;
    q[1] = wb * u;
    q[2] = wb * v;
    q[3] = wb * w;
    q[4] = wb * (p * ir / ph.R);
  }
  for (int o = 4; o > 0; o >>= 1)
    for (int v = 0; v < 5; v++) q[v] += __shfl_xor_sync(0xffffffffu, q[v], o);
  if (!live || b != 0 || mask == 0) return;
  const double ratio = sp->xi_node / sp->xi_probe;
  const double u = q[1] * ratio, v = q[2] * ratio, w = q[3] * ratio;
  const double r = q[0] / (ph.R * q[4]);
  const int node = sp->node;
  const long long id = cid(g, node % g.nx, (node / g.nx) % g.ny, node / (g.nx * g.ny));
  U.v[0][id] = r;
  U.v[1][id] = r * u;
  U.v[2][id] = r * v;
  U.v[3][id] = r * w;
  U.v[4][id] = q[0] / (ph.gamma - 1.0) + 0.5 * r * (u * u + v * v + w * w);
}

// Eq. 9 per triangle (tri: area per triangle; st: its probe): (-(p_s - p_inf) n + mu (u - (u.n) n) / xi) A
__global__ void __launch_bounds__(TB) k3_surface_force(Grid3 g, Phys3 ph, F5 U, const ibm_stencil3d *__restrict__ st,
                                                       const double *__restrict__ area, int ntri,
                                                       double *__restrict__ fout) {
  const int f = blockIdx.x * TB + threadIdx.x;
  if (f >= ntri) return;
  const ibm_stencil3d &s = st[f];
  double F[3] = {0.0, 0.0, 0.0};
  if (s.mask) {
    double qp[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = 0; b < 8; b++) {
      if (!(s.mask >> b & 1)) continue;
      const long long id = cid(g, s.i0 + (b & 1), s.j0 + (b >> 1 & 1), s.k0 + (b >> 2));
      const double r = U.v[0][id], ir = 1.0 / r;
      const double u = U.v[1][id] * ir, v = U.v[2][id] * ir, w = U.v[3][id] * ir;
      const double p = (ph.gamma - 1.0) * (U.v[4][id] - 0.5 * r * (u * u + v * v + w * w));
      qp[0] += s.w[b] * p;
      qp[1] += s.w[b] * u;
      qp[2] += s.w[b] * v;
      qp[3] += s.w[b] * w;
    }
    const double un = qp[1] * s.n[0] + qp[2] * s.n[1] + qp[3] * s.n[2];
    for (int a = 0; a < 3; a++) {
      const double tau = ph.mu * (qp[1 + a] - un * s.n[a]) / s.xi_probe;
      F[a] = (-(qp[0] - ph.pinf) * s.n[a] + tau) * area[f];
    }
  }
  for (int a = 0; a < 3; a++) fout[3 * f + a] = F[a];
}

// fixed-order sum of the per-triangle forces (one block: strided partial sums, then a tree)
__global__ void __launch_bounds__(TB) k3_force_sum(const double *__restrict__ fin, int ntri, double *__restrict__ out) {
  __shared__ double sh[3][TB];
  double s[3] = {0.0, 0.0, 0.0};
  for (int f = threadIdx.x; f < ntri; f += TB)
    for (int a = 0; a < 3; a++) s[a] += fin[3 * f + a];
  for (int a = 0; a < 3; a++) sh[a][threadIdx.x] = s[a];
  __syncthreads();
  for (int w = TB / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int a = 0; a < 3; a++) sh[a][threadIdx.x] += sh[a][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 3) out[threadIdx.x] = sh[threadIdx.x][0];
}

// end of step on the device: t += dt, last dt
__global__ void k3_step_end(const double *__restrict__ dtp, double *__restrict__ time) {
  const double dt = *dtp;
  time[0] = time[0] + dt;
  time[1] = dt;
}

// ---- FP32-bulk stages: values and fluxes in FP32 on perturbations from the free stream ------------------------
// The stage values are FP32 conserved perturbations U - U_inf: a mirror of the FP64 master U^n and the two
// intermediate stages.  Reconstruction, halos (the free stream is 0), primitives (rho', u', v', w', p', T') =
// (rho - 1, u - U_inf, ..., p - p_inf, T - 1), the CFL bound and the first two updates run in FP32; the fluxes
// are assembled so that no free-stream constant enters an FP32 sum: the pressure term as (p_half - p_inf) =
// p_inf (D_L + D_R - 1) + D_L p'_L + D_R p'_R, and the energy equation in the variable rho E - rho H_inf, whose
// flux is rho u H' (H' = H - H_inf); the updates restore L(rho E) = L' + H_inf L(rho).  FP64 appears only in the
// last stage, which accumulates its FP32 increment onto the master and refreshes the mirror from it.

struct P32 {
  float pinf, ipinf, gamma, gg, igm1, mu, kappa, ipr, u0[3], u2;  // gg = gamma / (gamma - 1), igm1 = 1 / (gamma - 1),
                                                                   // ipr = 1 / Pr, u2 = |U_inf|^2
  float ih[3], ih2;  // inverse spacings 1/dx, 1/dy, 1/dz and 1/dx^2 + 1/dy^2 + 1/dz^2
  float Hinf;        // free-stream total enthalpy
};

struct F5f {
  float *v[5];
};
struct F6f {
  float *v[6];  // rho', u', v', w', p', T'
};

// primitive perturbations of a conserved perturbation (drho, dm, dE) in FP32, free of cancellation:
//   u' = (dm - U_inf drho) / rho,  p' = (gamma - 1) (dE - (rho u'.(2 U_inf + u') + drho |U_inf|^2) / 2)
__device__ __forceinline__ void pert_prim(const P32 &c, float dr, const float dm[3], float dE, float &ir, float up[3],
                                          float &pp) {
  const float r = 1.0f + dr;
  ir = __fdividef(1.0f, r);
  float k = 0.0f;
  for (int a = 0; a < 3; a++) {
    up[a] = (dm[a] - c.u0[a] * dr) * ir;
    k += up[a] * (2.0f * c.u0[a] + up[a]);
  }
  pp = (c.gamma - 1.0f) * (dE - 0.5f * (r * k + dr * c.u2));
}

// FP32 perturbation sets of the FP64 master: S = U - U_inf over every cell (creation, ibm_case3d_set_state)
__global__ void __launch_bounds__(TC) k3_mirror32(Grid3 g, Phys3 ph, F5 U, F5f S) {
  const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y;
  if (x >= g.W || y >= g.H) return;
  const long long m = ((long long)blockIdx.z * g.H + y) * g.W + x;
  for (int v = 0; v < 5; v++) S.v[v][m] = (float)(U.v[v][m] - ph.Uinf[v]);
}

// primitive perturbations (rho', u', v', w', p', T') of an FP32 stage set, every cell (T' = (p'/p_inf - rho')/rho)
__global__ void __launch_bounds__(TC) k3_prim32(Grid3 g, P32 c, F5f S, F6f Q) {
  const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y;
  if (x >= g.W || y >= g.H) return;
  const long long m = ((long long)blockIdx.z * g.H + y) * g.W + x;
  const float dr = S.v[0][m], dm[3] = {S.v[1][m], S.v[2][m], S.v[3][m]}, dE = S.v[4][m];
  float ir, up[3], pp;
  pert_prim(c, dr, dm, dE, ir, up, pp);
  Q.v[0][m] = dr;
  Q.v[1][m] = up[0];
  Q.v[2][m] = up[1];
  Q.v[3][m] = up[2];
  Q.v[4][m] = pp;
  Q.v[5][m] = (pp * c.ipinf - dr) * ir;
}

// dt of the step from the CFL reduction (or the fixed step), once
__global__ void k3_dt(Phys3 ph, const unsigned long long *__restrict__ lmax, double *__restrict__ dt) {
  *dt = ph.dt_fixed > 0.0 ? ph.dt_fixed : ph.cfl / __longlong_as_double((long long)*lmax);
}

// CFL reduction of the FP32-bulk mode, in FP32 from the mirror of the master: each thread strides over z, the
// block reduces in shared memory and one atomic per block takes the maximum
__global__ void __launch_bounds__(TC) k3_lambda32(Grid3 g, P32 c, F5f M, const uint8_t *__restrict__ tags,
                                                  unsigned long long *__restrict__ lmax) {
  __shared__ float wmax[TC / 32];
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y;
  float lam = 0.0f;
  if (i < g.nx && j < g.ny) {
    for (int k = blockIdx.z; k < g.nz; k += gridDim.z) {
      if (tags[((long long)k * g.ny + j) * g.nx + i] != TAG_FLUID) continue;
      const long long m = cid(g, i, j, k);
      const float dr = M.v[0][m], dm[3] = {M.v[1][m], M.v[2][m], M.v[3][m]};
      float ir, up[3], pp;
      pert_prim(c, dr, dm, M.v[4][m], ir, up, pp);
      const float p = c.pinf + pp, c2 = c.gamma * p * ir, cs = c2 * rsqrtf(c2);
      const float l = (fabsf(c.u0[0] + up[0]) + cs) * c.ih[0] + (fabsf(c.u0[1] + up[1]) + cs) * c.ih[1] +
                      (fabsf(c.u0[2] + up[2]) + cs) * c.ih[2] + (2.0f * c.gamma * c.mu * c.ipr * ir) * c.ih2;
      lam = fmaxf(lam, l);
    }
  }
  for (int o = 16; o > 0; o >>= 1) lam = fmaxf(lam, __shfl_xor_sync(0xffffffffu, lam, o));
  const int tid = threadIdx.y * BX + threadIdx.x;
  if ((tid & 31) == 0) wmax[tid >> 5] = lam;
  __syncthreads();
  if (tid == 0) {
    float b = wmax[0];
    for (int w = 1; w < TC / 32; w++) b = fmaxf(b, wmax[w]);
    if (b > 0.0f) atomicMax(lmax, (unsigned long long)__double_as_longlong((double)b));
  }
}

// Sec. 4.4-4.6 and Sec. 5 on an FP32 stage set (the FP64 kernel's rule in perturbation form): eight lanes per
// node, one cube corner each, sums of (p', u', v', w', T') by a fixed shuffle tree; the node's conserved
// perturbation follows from p = p_inf + p', u = (U_inf + u') xi_node / xi_probe, T = 1 + T'.  With master set,
// the node's value is also written to the FP64 master (the first stage's reconstruction, from U^n).
__global__ void __launch_bounds__(128) k3_reconstruct32(Grid3 g, Phys3 ph, P32 c, F5f S,
                                                        const ibm_stencil3d *__restrict__ st, int first, int count,
                                                        F5 A, int master) {
  const int t = blockIdx.x * 128 + threadIdx.x;
  const int e = t >> 3, b = t & 7;
  const bool live = e < count;
  const ibm_stencil3d *sp = st + first + (live ? e : 0);
  const int mask = live ? sp->mask : 0;
  float q[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
  if (mask >> b & 1) {
    const long long id = cid(g, sp->i0 + (b & 1), sp->j0 + (b >> 1 & 1), sp->k0 + (b >> 2));
    const float dr = S.v[0][id], dm[3] = {S.v[1][id], S.v[2][id], S.v[3][id]};
    float ir, up[3], pp;
    pert_prim(c, dr, dm, S.v[4][id], ir, up, pp);
    const float wb = (float)sp->w[b];
    q[0] = wb * pp;
    q[1] = wb * up[0];
    q[2] = wb * up[1];
    q[3] = wb * up[2];
    q[4] = wb * ((pp * c.ipinf - dr) * ir);
  }
  for (int o = 4; o > 0; o >>= 1)
    for (int v = 0; v < 5; v++) q[v] += __shfl_xor_sync(0xffffffffu, q[v], o);
  if (!live || b != 0 || mask == 0) return;
  const float ratio = (float)(sp->xi_node / sp->xi_probe);
  const float pp = q[0], Tp = q[4];
  const float dr = (pp * c.ipinf - Tp) * __fdividef(1.0f, 1.0f + Tp);  // rho - 1 = (p / p_inf) / (1 + T') - 1
  float out[5], k = 0.0f;
  out[0] = dr;
  for (int a = 0; a < 3; a++) {
    const float up = ratio * (c.u0[a] + q[1 + a]) - c.u0[a];
    out[1 + a] = up + dr * (c.u0[a] + up);  // rho u - U_inf
    k += up * (2.0f * c.u0[a] + up);
  }
  out[4] = pp * c.igm1 + 0.5f * ((1.0f + dr) * k + dr * c.u2);
  const int node = sp->node;
  const long long id = cid(g, node % g.nx, (node / g.nx) % g.ny, node / (g.nx * g.ny));
  for (int v = 0; v < 5; v++) S.v[v][id] = out[v];
  if (master)
    for (int v = 0; v < 5; v++) A.v[v][id] = ph.Uinf[v] + (double)out[v];
}

// domain halos of an FP32 stage set (perturbations: the free stream is 0), the FP64 kernel's closed form
__global__ void __launch_bounds__(TB) k3_halo32(Grid3 g, F5f U) {
  const int t = blockIdx.x * TB + threadIdx.x;
  const int nzs = 2 * NG * g.W * g.H, nys = 2 * NG * g.nz * g.W, nxs = 2 * NG * g.nz * g.ny;
  int x, y, z;
  if (t < nzs) {
    const int zz = t / (g.W * g.H), rem = t - zz * (g.W * g.H);
    z = zz < NG ? zz : g.nz + zz;
    y = rem / g.W;
    x = rem - y * g.W;
  } else if (t < nzs + nys) {
    const int u = t - nzs, zz = u / (2 * NG * g.W), rem = u - zz * (2 * NG * g.W), yy = rem / g.W;
    z = NG + zz;
    y = yy < NG ? yy : g.ny + yy;
    x = rem - yy * g.W;
  } else if (t < nzs + nys + nxs) {
    const int u = t - nzs - nys, zz = u / (2 * NG * g.ny), rem = u - zz * (2 * NG * g.ny), yy = rem / (2 * NG);
    const int xx = rem - yy * (2 * NG);
    z = NG + zz;
    y = NG + yy;
    x = xx < NG ? xx : g.nx + xx;
  } else {
    return;
  }
  const long long m = ((long long)z * g.H + y) * g.W + x;
  const int I[3] = {x - NG, y - NG, z - NG};
  const int n[3] = {g.nx, g.ny, g.nz};
  int S[3];
  bool fs = false;
  for (int a = 0; a < 3; a++) {
    S[a] = I[a];
    if (I[a] >= 0 && I[a] < n[a]) continue;
    const int bc = g.bc[2 * a + (I[a] < 0 ? 0 : 1)];
    if (bc == IBM_BC_PERIODIC) S[a] = I[a] < 0 ? I[a] + n[a] : I[a] - n[a];
    else if (bc == IBM_BC_OUTFLOW) S[a] = I[a] < 0 ? 0 : n[a] - 1;
    else fs = true;
  }
  if (fs) {
    for (int v = 0; v < 5; v++) U.v[v][m] = 0.0f;
  } else {
    const long long src = cid(g, S[0], S[1], S[2]);
    for (int v = 0; v < 5; v++) U.v[v][m] = U.v[v][src];
  }
}

__device__ __forceinline__ float weno5f(float f0, float f1, float f2, float f3, float f4) {
  const float eps = 1e-6f;
  float a = f0 - 2.0f * f1 + f2, b = f0 - 4.0f * f1 + 3.0f * f2;
  const float b0 = (13.0f / 12.0f) * a * a + 0.25f * b * b;
  a = f1 - 2.0f * f2 + f3;
  b = f1 - f3;
  const float b1 = (13.0f / 12.0f) * a * a + 0.25f * b * b;
  a = f2 - 2.0f * f3 + f4;
  b = 3.0f * f2 - 4.0f * f3 + f4;
  const float b2 = (13.0f / 12.0f) * a * a + 0.25f * b * b;
  const float q0 = (2.0f * f0 - 7.0f * f1 + 11.0f * f2) * (1.0f / 6.0f);
  const float q1 = (-f1 + 5.0f * f2 + 2.0f * f3) * (1.0f / 6.0f);
  const float q2 = (2.0f * f2 + 5.0f * f3 - f4) * (1.0f / 6.0f);
  // alpha_k = d_k / (eps + beta_k)^2 through FP32 reciprocals (in range for beta_k up to ~1e19)
  const float e0 = eps + b0, e1 = eps + b1, e2 = eps + b2;
  const float i0 = __fdividef(1.0f, e0 * e0), i1 = __fdividef(1.0f, e1 * e1), i2 = __fdividef(1.0f, e2 * e2);
  const float a0 = 0.1f * i0, a1 = 0.6f * i1, a2 = 0.3f * i2;
  return __fdividef(a0 * q0 + a1 * q1 + a2 * q2, a0 + a1 + a2);
}

// LDFSS(0) (Mr = 1) on perturbation states q' = (rho', u', v', w', p'); F = mass, momentum less p_inf n,
// rho u H'
template <int DIR>
__device__ __forceinline__ void ldfss32(const float qL[5], const float qR[5], const P32 &c, float F[5]) {
  const float rL = 1.0f + qL[0], rR = 1.0f + qR[0];
  const float irL = __fdividef(1.0f, rL), irR = __fdividef(1.0f, rR);
  const float pL = c.pinf + qL[4], pR = c.pinf + qR[4];
  const float c2L = c.gamma * pL * irL, c2R = c.gamma * pR * irR;
  const float cL = c2L * rsqrtf(c2L), cR = c2R * rsqrtf(c2R);  // sound speeds (approximate square roots)
  float uL[3], uR[3];
  for (int a = 0; a < 3; a++) {
    uL[a] = c.u0[a] + qL[1 + a];
    uR[a] = c.u0[a] + qR[1 + a];
  }
  // H' = gamma/(gamma-1) (p / rho - p_inf) + (|u|^2 - |U_inf|^2) / 2
  float kL = 0.0f, kR = 0.0f;
  for (int a = 0; a < 3; a++) {
    kL += qL[1 + a] * (2.0f * c.u0[a] + qL[1 + a]);
    kR += qR[1 + a] * (2.0f * c.u0[a] + qR[1 + a]);
  }
  const float HL = c.gg * (qL[4] - c.pinf * qL[0]) * irL + 0.5f * kL;
  const float HR = c.gg * (qR[4] - c.pinf * qR[0]) * irR + 0.5f * kR;
  const float unL = uL[DIR], unR = uR[DIR];
  const float cs = 0.5f * (cL + cR), ics = __fdividef(1.0f, cs);
  const float ML = unL * ics, MR = unR * ics;
  const float aL = ML >= 0.0f ? 1.0f : 0.0f, aR = MR >= 0.0f ? 0.0f : 1.0f;
  const float bL = -fmaxf(1.0f - floorf(fabsf(ML)), 0.0f), bR = -fmaxf(1.0f - floorf(fabsf(MR)), 0.0f);
  const float MpL = 0.25f * (ML + 1.0f) * (ML + 1.0f);
  const float MmR = -0.25f * (MR - 1.0f) * (MR - 1.0f);
  const float CVL = aL * (1.0f + bL) * ML - bL * MpL;
  const float CVR = aR * (1.0f + bR) * MR - bR * MmR;
  const float m2 = 0.5f * (ML * ML + MR * MR);
  const float sq = (m2 > 0.0f ? m2 * rsqrtf(m2) : 0.0f) - 1.0f;
  const float Mh = 0.25f * bL * bR * sq * sq;
  const float dp = qL[4] - qR[4], adp = fabsf(dp), ic2 = 0.5f * ics * ics;
  const float MhP = Mh * (1.0f - (dp + adp) * ic2 * irL);
  const float MhM = Mh * (1.0f - (-dp + adp) * ic2 * irR);
  const float Cp = CVL - MhP, Cm = CVR + MhM;
  const float PpL = 0.25f * (ML + 1.0f) * (ML + 1.0f) * (2.0f - ML);
  const float PmR = 0.25f * (MR - 1.0f) * (MR - 1.0f) * (2.0f + MR);
  const float DL = aL * (1.0f + bL) - bL * PpL;
  const float DR = aR * (1.0f + bR) - bR * PmR;
  const float mL = rL * cs * Cp, mR = rR * cs * Cm;
  const float php = c.pinf * ((DL + DR) - 1.0f) + (DL * qL[4] + DR * qR[4]);
  F[0] = mL + mR;
  for (int a = 0; a < 3; a++) F[1 + a] = mL * uL[a] + mR * uR[a];
  F[1 + DIR] += php;
  F[4] = mL * HL + mR * HR;
}

template <int DIR>
__global__ void __launch_bounds__(TC) k3_flux32(Grid3 g, P32 c, F6f Q, F5f Fo) {
  // faces i + 1/2 (DIR 0) for i in [-1, nx - 1], likewise along y and z; one thread per face
  int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= g.nx + (DIR == 0) || j >= g.ny + (DIR == 1)) return;
  if (DIR == 0) i -= 1;
  if (DIR == 1) j -= 1;
  if (DIR == 2) k -= 1;
  const long long st = DIR == 0 ? 1 : DIR == 1 ? (long long)g.W : g.plane;
  const long long a = cid(g, i, j, k), b = a + st;
  float qL[5], qR[5];
  for (int v = 0; v < 5; v++) {
    const float *q = Q.v[v];
    const float f0 = q[a - 2 * st], f1 = q[a - st], f2 = q[a], f3 = q[b], f4 = q[b + st], f5 = q[b + 2 * st];
    qL[v] = weno5f(f0, f1, f2, f3, f4);
    qR[v] = weno5f(f5, f4, f3, f2, f1);
  }
  if (!(1.0f + qL[0] > 0.0f) || !(c.pinf + qL[4] > 0.0f) || !(1.0f + qR[0] > 0.0f) || !(c.pinf + qR[4] > 0.0f)) {
    for (int v = 0; v < 5; v++) {
      qL[v] = Q.v[v][a];
      qR[v] = Q.v[v][b];
    }
  }
  float F[5];
  ldfss32<DIR>(qL, qR, c, F);
  if (c.mu > 0.0f) {
    const int t1 = DIR == 0 ? 1 : 0, t2 = DIR == 2 ? 1 : 2;
    const long long s1 = t1 == 0 ? 1 : (long long)g.W, s2 = t2 == 1 ? (long long)g.W : g.plane;
    const float in = c.ih[DIR], i1 = 0.25f * c.ih[t1], i2 = 0.25f * c.ih[t2];
    float G[3][3];
    for (int cc = 0; cc < 3; cc++) {
      const float *q = Q.v[1 + cc];
      G[cc][DIR] = (q[b] - q[a]) * in;
      G[cc][t1] = (q[a + s1] - q[a - s1] + q[b + s1] - q[b - s1]) * i1;
      G[cc][t2] = (q[a + s2] - q[a - s2] + q[b + s2] - q[b - s2]) * i2;
    }
    const float div = G[0][0] + G[1][1] + G[2][2];
    float tau[3];
    for (int cc = 0; cc < 3; cc++) tau[cc] = c.mu * (G[cc][DIR] + G[DIR][cc]);
    tau[DIR] = c.mu * (2.0f * G[DIR][DIR] - (2.0f / 3.0f) * div);
    const float qn = -c.kappa * (Q.v[5][b] - Q.v[5][a]) * in;
    float work = 0.0f;
    for (int cc = 0; cc < 3; cc++) {
      F[1 + cc] -= tau[cc];
      work += (c.u0[cc] + 0.5f * (Q.v[1 + cc][a] + Q.v[1 + cc][b])) * tau[cc];
    }
    F[4] -= work - qn;
  }
  for (int v = 0; v < 5; v++) Fo.v[v][a] = F[v];
}

// SSP-RK3 stages 1 and 2 on the fluid cells in FP32 from the flux divergence (L(rho E) = L' + H_inf L(rho)),
// on perturbations: out = M + dt L, M + ((In - M) + dt L) / 4, with M the mirror of U^n
__device__ __forceinline__ void flux_div32(const Grid3 &g, const P32 &c, const F5f &Fx, const F5f &Fy, const F5f &Fz,
                                           long long m, float L[5]) {
  const float ix = c.ih[0], iy = c.ih[1], iz = c.ih[2], Hinf = c.Hinf;
  for (int v = 0; v < 5; v++)
    L[v] = -((Fx.v[v][m] - Fx.v[v][m - 1]) * ix + (Fy.v[v][m] - Fy.v[v][m - g.W]) * iy +
             (Fz.v[v][m] - Fz.v[v][m - g.plane]) * iz);
  L[4] += Hinf * L[0];
}

__global__ void __launch_bounds__(TC) k3_update32(Grid3 g, P32 c, int stage, F5f Fx, F5f Fy, F5f Fz, F5f M,
                                                  F5f In, F5f Out, const uint8_t *__restrict__ tags,
                                                  const double *__restrict__ dtp) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  if (tags[((long long)k * g.ny + j) * g.nx + i] != TAG_FLUID) return;
  const long long m = cid(g, i, j, k);
  const float dt = (float)*dtp;
  float L[5];
  flux_div32(g, c, Fx, Fy, Fz, m, L);
  for (int v = 0; v < 5; v++) {
    const float mv = M.v[v][m];
    Out.v[v][m] = stage == 1 ? mv + dt * L[v] : mv + 0.25f * ((In.v[v][m] - mv) + dt * L[v]);
  }
}

// SSP-RK3 stage 3: the increment 2/3 ((In - M) + dt L) in FP32, accumulated onto the FP64 master, whose new
// value refreshes the mirror
__global__ void __launch_bounds__(TC) k3_update32_last(Grid3 g, Phys3 ph, P32 c, F5f Fx, F5f Fy, F5f Fz, F5 A,
                                                       F5f M, F5f In, const uint8_t *__restrict__ tags,
                                                       const double *__restrict__ dtp) {
  const int i = blockIdx.x * BX + threadIdx.x, j = blockIdx.y * BY + threadIdx.y, k = blockIdx.z;
  if (i >= g.nx || j >= g.ny) return;
  if (tags[((long long)k * g.ny + j) * g.nx + i] != TAG_FLUID) return;
  const long long m = cid(g, i, j, k);
  const float dt = (float)*dtp;
  float L[5];
  flux_div32(g, c, Fx, Fy, Fz, m, L);
  for (int v = 0; v < 5; v++) {
    const float d = (2.0f / 3.0f) * ((In.v[v][m] - M.v[v][m]) + dt * L[v]);
    const double a = A.v[v][m] + (double)d;
    A.v[v][m] = a;
    M.v[v][m] = (float)(a - ph.Uinf[v]);
  }
}

inline unsigned nblk(long long n) { return (unsigned)((n + TB - 1) / TB); }
inline dim3 cells(int ex, int ey, int ez) { return dim3((ex + BX - 1) / BX, (ey + BY - 1) / BY, ez); }
const dim3 CB(BX, BY, 1);

}  // namespace

struct ibm_case3d {
  Grid3 g{};
  Phys3 ph{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  ibm_body3d *body = nullptr;
  int ntri = 0;
  char *mem = nullptr;  // one allocation for every array below
  F5 A{}, B{}, C{}, Fx{}, Fy{}, Fz{};
  F6 Q{};
  uint8_t *tags = nullptr;        // the body's tags, or the case's own (all fluid) without a body
  uint8_t *own_tags = nullptr;
  ibm_stencil3d *st = nullptr;    // listed nodes
  ibm_stencil3d *sst = nullptr;   // force probes, one per triangle
  double *tri = nullptr;          // per triangle: centroid, normal (6 doubles), then the areas
  double *fbuf = nullptr;         // per-triangle forces, then the summed force (3 doubles)
  unsigned long long *lmax = nullptr;
  double *time = nullptr;         // t, last dt
  double *dt = nullptr;           // dt of the current step
  int *nerr = nullptr;
  int counts[4] = {0, 0, 0, 0};
  double ref_area = 1.0;
  int precision = IBM_PREC_FP64;
  P32 p32{};
  double Hinf = 0.0;
  // FP32-bulk views into the storage of the FP64 stage, primitive and flux arrays: the mirror of the master
  // and the two intermediate stage sets (perturbations), primitives, face fluxes
  F5f mirror{}, s1{}, s2{}, fx32{}, fy32{}, fz32{};
  F6f q32{};
  int64_t launches = 0;
};

static ibm_status cfail(cudaError_t e) { return ibm__noalloc_fail(IBM_ECUDA, cudaGetErrorString(e)); }

extern "C" ibm_status ibm_case3d_destroy(ibm_case3d *c) {
  if (!c) return IBM_OK;
  if (c->stream) cudaStreamSynchronize(c->stream);
  ibm_body3d_destroy(c->body);
  cudaFree(c->mem);
  cudaFree(c->own_tags);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
  return IBM_OK;
}

extern "C" ibm_status ibm_case3d_create(const double *verts, int nverts, const int32_t *tris, int ntris,
                                        const ibm_flow3d *fl, void *cuda_stream, ibm_case3d **out) {
  if (!out || !fl) return ibm__noalloc_fail(IBM_EINVAL, "ibm_case3d_create: NULL argument");
  *out = nullptr;
  if (fl->nx < 4 || fl->ny < 4 || fl->nz < 4) return ibm__noalloc_fail(IBM_EINVAL, "ibm_case3d_create: fewer than 4 cells along an axis");
  for (int a = 0; a < 3; a++)
    if (!(fl->hi[a] > fl->lo[a])) return ibm__noalloc_fail(IBM_EINVAL, "ibm_case3d_create: empty domain");
  for (int k = 0; k < 6; k++)
    if (fl->bc[k] < IBM_BC_FREESTREAM || fl->bc[k] > IBM_BC_PERIODIC) return ibm__noalloc_fail(IBM_EINVAL, "ibm_case3d_create: bad boundary condition");
  for (int a = 0; a < 3; a++)
    if ((fl->bc[2 * a] == IBM_BC_PERIODIC) != (fl->bc[2 * a + 1] == IBM_BC_PERIODIC))
      return ibm__noalloc_fail(IBM_EINVAL, "ibm_case3d_create: periodic on one side of an axis only");
  if (!(fl->mach > 0.0) || !(fl->gamma > 1.0) || !(fl->prandtl > 0.0) || !(fl->ref_area > 0.0) ||
      !(fl->dt_fixed > 0.0 || fl->cfl > 0.0))
    return ibm__noalloc_fail(IBM_EINVAL, "ibm_case3d_create: bad flow parameters");
  if (ntris < 0 || (ntris > 0 && (!verts || !tris))) return ibm__noalloc_fail(IBM_EINVAL, "ibm_case3d_create: bad mesh");
  const long long nn = (long long)fl->nx * fl->ny * fl->nz;
  if (nn > (1LL << 31) - 1) return ibm__noalloc_fail(IBM_EINVAL, "ibm_case3d_create: more than 2^31 - 1 cells");
  if (fl->precision != IBM_PREC_FP64 && fl->precision != IBM_PREC_FP32_BULK)
    return ibm__noalloc_fail(IBM_EINVAL, "ibm_case3d_create: unknown precision");
  ibm_case3d *c = new ibm_case3d();
  c->ref_area = fl->ref_area;
  c->precision = fl->precision;
  Grid3 &g = c->g;
  g.nx = fl->nx;
  g.ny = fl->ny;
  g.nz = fl->nz;
  g.W = g.nx + 2 * NG;
  g.H = g.ny + 2 * NG;
  g.D = g.nz + 2 * NG;
  g.plane = (long long)g.W * g.H;
  g.ncell = g.plane * g.D;
  g.dx = (fl->hi[0] - fl->lo[0]) / fl->nx;
  g.dy = (fl->hi[1] - fl->lo[1]) / fl->ny;
  g.dz = (fl->hi[2] - fl->lo[2]) / fl->nz;
  g.idx = 1.0 / g.dx;
  g.idy = 1.0 / g.dy;
  g.idz = 1.0 / g.dz;
  for (int a = 0; a < 3; a++) g.lo[a] = fl->lo[a];
  for (int k = 0; k < 6; k++) g.bc[k] = fl->bc[k];
  Phys3 &ph = c->ph;
  ph.gamma = fl->gamma;
  ph.pinf = 1.0 / (fl->gamma * fl->mach * fl->mach);
  ph.R = ph.pinf;
  ph.mu = fl->re > 0.0 ? 1.0 / fl->re : 0.0;
  ph.kappa = ph.mu * (fl->gamma * ph.R / (fl->gamma - 1.0)) / fl->prandtl;
  ph.prandtl = fl->prandtl;
  ph.cfl = fl->cfl;
  ph.dt_fixed = fl->dt_fixed;
  const double u = fl->uinf[0], v = fl->uinf[1], w = fl->uinf[2];
  ph.Uinf[0] = 1.0;
  ph.Uinf[1] = u;
  ph.Uinf[2] = v;
  ph.Uinf[3] = w;
  ph.Uinf[4] = ph.pinf / (fl->gamma - 1.0) + 0.5 * (u * u + v * v + w * w);
  c->Hinf = fl->gamma / (fl->gamma - 1.0) * ph.pinf + 0.5 * (u * u + v * v + w * w);
  c->p32.pinf = (float)ph.pinf;
  c->p32.ipinf = (float)(1.0 / ph.pinf);
  c->p32.igm1 = (float)(1.0 / (fl->gamma - 1.0));
  c->p32.u2 = (float)(u * u + v * v + w * w);
  c->p32.Hinf = (float)c->Hinf;
  c->p32.ih[0] = (float)g.idx;
  c->p32.ih[1] = (float)g.idy;
  c->p32.ih[2] = (float)g.idz;
  c->p32.ih2 = (float)(g.idx * g.idx + g.idy * g.idy + g.idz * g.idz);
  c->p32.ipr = (float)(1.0 / fl->prandtl);
  c->p32.gamma = (float)fl->gamma;
  c->p32.gg = (float)(fl->gamma / (fl->gamma - 1.0));
  c->p32.mu = (float)ph.mu;
  c->p32.kappa = (float)ph.kappa;
  for (int a = 0; a < 3; a++) c->p32.u0[a] = (float)fl->uinf[a];
  cudaError_t e = cudaSuccess;
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
  } else {
    e = cudaStreamCreate(&c->stream);  // synchronises with the legacy default stream, as a 2-D case's own
    c->own_stream = e == cudaSuccess;
    if (e != cudaSuccess) {
      delete c;
      return cfail(e);
    }
  }
  // geometry: classification, tags, lists and stencils on the case stream
  const double h = std::sqrt(g.dx * g.dx + g.dy * g.dy + g.dz * g.dz);
  const double dmin = std::fmin(g.dx, std::fmin(g.dy, g.dz));
  int cap = 0;
  c->ntri = ntris;
  if (ntris > 0) {
    ibm_status s = ibm_body3d_create(verts, nverts, tris, ntris, c->stream, &c->body);
    if (s == IBM_OK) {
      ibm_grid3d lg;
      lg.nx = g.nx;
      lg.ny = g.ny;
      lg.nz = g.nz;
      for (int a = 0; a < 3; a++) {
        lg.lo[a] = fl->lo[a];
        lg.hi[a] = fl->hi[a];
      }
      s = ibm_body3d_classify(c->body, &lg);
    }
    if (s != IBM_OK) {
      ibm_case3d_destroy(c);
      return s;
    }
    cap = ibm__body3d_capacity(c->body);
  }
  // one allocation: 3 x 5 state arrays, 6 primitive arrays, 3 x 5 flux arrays, stencils, triangles, forces
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t arr = up((size_t)g.ncell * sizeof(double));
  const size_t s_st = up((size_t)std::max(cap, 1) * sizeof(ibm_stencil3d));
  const size_t s_sst = up((size_t)std::max(ntris, 1) * sizeof(ibm_stencil3d));
  const size_t s_tri = up((size_t)std::max(ntris, 1) * 7 * sizeof(double));
  const size_t s_f = up(((size_t)std::max(ntris, 1) * 3 + 3) * sizeof(double));
  const size_t total = arr * 36 + s_st + s_sst + s_tri + s_f + 256 * 4;
  e = cudaMalloc(&c->mem, total);
  if (e != cudaSuccess) {
    ibm_case3d_destroy(c);
    return ibm__noalloc_fail(IBM_ENOMEM, "ibm_case3d_create: device allocation failed");
  }
  char *p = c->mem;
  auto take = [&](size_t n) {
    char *q = p;
    p += n;
    return q;
  };
  for (int v = 0; v < 5; v++) {
    c->A.v[v] = (double *)take(arr);
    c->B.v[v] = (double *)take(arr);
    c->C.v[v] = (double *)take(arr);
    c->Fx.v[v] = (double *)take(arr);
    c->Fy.v[v] = (double *)take(arr);
    c->Fz.v[v] = (double *)take(arr);
  }
  for (int v = 0; v < 6; v++) c->Q.v[v] = (double *)take(arr);
  c->st = (ibm_stencil3d *)take(s_st);
  c->sst = (ibm_stencil3d *)take(s_sst);
  c->tri = (double *)take(s_tri);
  c->fbuf = (double *)take(s_f);
  c->lmax = (unsigned long long *)take(256);
  c->time = (double *)take(256);
  c->nerr = (int *)take(256);
  c->dt = (double *)take(256);
  // free stream everywhere (halos and solid cells included)
  {
    std::vector<double> fsv((size_t)g.ncell);
    for (int v = 0; v < 5 && e == cudaSuccess; v++) {
      std::fill(fsv.begin(), fsv.end(), ph.Uinf[v]);
      e = cudaMemcpyAsync(c->A.v[v], fsv.data(), (size_t)g.ncell * sizeof(double), cudaMemcpyHostToDevice, c->stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(c->B.v[v], c->A.v[v], (size_t)g.ncell * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(c->C.v[v], c->A.v[v], (size_t)g.ncell * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);  // fsv is reused
    }
  }
  for (int v = 0; v < 5; v++) {
    c->mirror.v[v] = (float *)c->B.v[v];
    c->s2.v[v] = (float *)c->B.v[v] + g.ncell;
    c->s1.v[v] = (float *)c->C.v[v];
    c->fx32.v[v] = (float *)c->Fx.v[v];
    c->fy32.v[v] = (float *)c->Fy.v[v];
    c->fz32.v[v] = (float *)c->Fz.v[v];
  }
  for (int v = 0; v < 6; v++) c->q32.v[v] = (float *)c->Q.v[v];
  if (e == cudaSuccess && c->precision == IBM_PREC_FP32_BULK) {
    // all three FP32 sets start as the master's perturbation (solid cells away from the body keep it)
    const dim3 ball = cells(g.W, g.H, g.D);
    k3_mirror32<<<ball, CB, 0, c->stream>>>(g, ph, c->A, c->mirror);
    k3_mirror32<<<ball, CB, 0, c->stream>>>(g, ph, c->A, c->s1);
    k3_mirror32<<<ball, CB, 0, c->stream>>>(g, ph, c->A, c->s2);
    c->launches += 3;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(c->time, 0, 256, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->nerr, 0, 256, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->lmax, 0, 256, c->stream);
  if (e != cudaSuccess) {
    ibm_case3d_destroy(c);
    return cfail(e);
  }
  if (ntris > 0) {
    // per triangle on the host: centroid, unit normal (the cross product of the edges from the first vertex),
    // area
    std::vector<double> td((size_t)ntris * 7);
    for (int f = 0; f < ntris; f++) {
      const double *Av = verts + 3 * tris[3 * f], *Bv = verts + 3 * tris[3 * f + 1], *Cv = verts + 3 * tris[3 * f + 2];
      double e1[3], e2[3], cr[3];
      for (int a = 0; a < 3; a++) {
        e1[a] = Bv[a] - Av[a];
        e2[a] = Cv[a] - Av[a];
        td[(size_t)6 * f + a] = (Av[a] + Bv[a] + Cv[a]) / 3.0;
      }
      cr[0] = e1[1] * e2[2] - e1[2] * e2[1];
      cr[1] = e1[2] * e2[0] - e1[0] * e2[2];
      cr[2] = e1[0] * e2[1] - e1[1] * e2[0];
      const double len = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
      for (int a = 0; a < 3; a++) td[(size_t)6 * f + 3 + a] = cr[a] / len;
      td[(size_t)6 * ntris + f] = 0.5 * len;
    }
    e = cudaMemcpyAsync(c->tri, td.data(), td.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
      ibm_case3d_destroy(c);
      return cfail(e);
    }
    const int *dcounts = nullptr;
    const uint8_t *dtags = nullptr;
    ibm_status s = ibm__body3d_stencils(c->body, h, dmin, c->st, c->nerr, &dtags, &dcounts, &cap);
    if (s == IBM_OK) s = ibm__surface3d_stencils(c->body, c->tri, ntris, h, dmin, c->sst);
    if (s != IBM_OK) {
      ibm_case3d_destroy(c);
      return s;
    }
    c->tags = (uint8_t *)dtags;
    int herr = 0;
    e = cudaMemcpyAsync(c->counts, dcounts, sizeof(c->counts), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, c->nerr, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
      ibm_case3d_destroy(c);
      return cfail(e);
    }
    c->launches += 7;
    if ((long long)c->counts[0] + c->counts[1] + c->counts[2] + c->counts[3] > cap) {
      ibm_case3d_destroy(c);
      return ibm__noalloc_fail(IBM_ECAPACITY, "ibm_case3d_create: more listed nodes than the capacity");
    }
    if (herr > 0) {
      ibm_case3d_destroy(c);
      return ibm__noalloc_fail(IBM_ESTENCIL, "ibm_case3d_create: a listed node found no valid probe corner");
    }
  } else {
    e = cudaMalloc(&c->own_tags, (size_t)nn);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->own_tags, 0, (size_t)nn, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
      ibm_case3d_destroy(c);
      return cfail(e);
    }
    c->tags = c->own_tags;
  }
  *out = c;
  return IBM_OK;
}

extern "C" ibm_status ibm_case3d_step(ibm_case3d *c, int nsteps) {
  if (!c || nsteps < 0) return ibm__noalloc_fail(IBM_EINVAL, "ibm_case3d_step: bad argument");
  const Grid3 &g = c->g;
  const Phys3 &ph = c->ph;
  const int nib = c->counts[0], ngh = c->counts[1] + c->counts[2] + c->counts[3];
  cudaStream_t s = c->stream;
  const bool f32 = c->precision == IBM_PREC_FP32_BULK;
  const dim3 bx = cells(g.nx + 1, g.ny, g.nz), by = cells(g.nx, g.ny + 1, g.nz), bz = cells(g.nx, g.ny, g.nz + 1);
  const dim3 ball = cells(g.W, g.H, g.D), bint = cells(g.nx, g.ny, g.nz);
  const unsigned bhalo = nblk(2LL * NG * ((long long)g.W * g.H + (long long)g.nz * g.W + (long long)g.nz * g.ny));
  // eight lanes per listed node (one cube corner each), 16 nodes per block
  const unsigned bib = (unsigned)((nib + 15) / 16), bgh = (unsigned)((ngh + 15) / 16);
  for (int it = 0; it < nsteps; it++) {
    if (ph.dt_fixed <= 0.0) {
      cudaMemsetAsync(c->lmax, 0, sizeof(unsigned long long), s);
      if (f32) k3_lambda32<<<cells(g.nx, g.ny, std::min(g.nz, 8)), CB, 0, s>>>(g, c->p32, c->mirror, c->tags, c->lmax);
      else k3_lambda<<<bint, CB, 0, s>>>(g, ph, c->A, c->tags, c->lmax);
      c->launches++;
    }
    k3_dt<<<1, 1, 0, s>>>(ph, c->lmax, c->dt);
    c->launches++;
    if (f32) {
      // FP32 stage sets: the mirror M of U^n, U^1, U^2 (perturbations); FP64 only in the last stage's
      // accumulation onto the master
      const F5f in[3] = {c->mirror, c->s1, c->s2};
      for (int k = 0; k < 3; k++) {
        if (nib) k3_reconstruct32<<<bib, 128, 0, s>>>(g, ph, c->p32, in[k], c->st, 0, nib, c->A, k == 0);
        if (ngh) k3_reconstruct32<<<bgh, 128, 0, s>>>(g, ph, c->p32, in[k], c->st, nib, ngh, c->A, k == 0);
        k3_halo32<<<bhalo, TB, 0, s>>>(g, in[k]);
        k3_prim32<<<ball, CB, 0, s>>>(g, c->p32, in[k], c->q32);
        k3_flux32<0><<<bx, CB, 0, s>>>(g, c->p32, c->q32, c->fx32);
        k3_flux32<1><<<by, CB, 0, s>>>(g, c->p32, c->q32, c->fy32);
        k3_flux32<2><<<bz, CB, 0, s>>>(g, c->p32, c->q32, c->fz32);
        if (k < 2)
          k3_update32<<<bint, CB, 0, s>>>(g, c->p32, k + 1, c->fx32, c->fy32, c->fz32, c->mirror, in[k],
                                          k == 0 ? c->s1 : c->s2, c->tags, c->dt);
        else
          k3_update32_last<<<bint, CB, 0, s>>>(g, ph, c->p32, c->fx32, c->fy32, c->fz32, c->A, c->mirror,
                                               in[k], c->tags, c->dt);
        c->launches += 6 + (nib ? 1 : 0) + (ngh ? 1 : 0);
      }
    } else {
      F5 in[3] = {c->A, c->B, c->C}, out[3] = {c->B, c->C, c->A};
      for (int k = 0; k < 3; k++) {
        if (nib) k3_reconstruct<<<bib, 128, 0, s>>>(g, ph, in[k], c->st, 0, nib);
        if (ngh) k3_reconstruct<<<bgh, 128, 0, s>>>(g, ph, in[k], c->st, nib, ngh);
        k3_halo<<<bhalo, TB, 0, s>>>(g, ph, in[k]);
        k3_prim<<<ball, CB, 0, s>>>(g, ph, in[k], c->Q);
        k3_flux<0><<<bx, CB, 0, s>>>(g, ph, c->Q, c->Fx);
        k3_flux<1><<<by, CB, 0, s>>>(g, ph, c->Q, c->Fy);
        k3_flux<2><<<bz, CB, 0, s>>>(g, ph, c->Q, c->Fz);
        k3_update<<<bint, CB, 0, s>>>(g, k + 1, c->Fx, c->Fy, c->Fz, c->A, in[k], out[k], c->tags, c->dt);
        c->launches += 6 + (nib ? 1 : 0) + (ngh ? 1 : 0);
      }
    }
    k3_step_end<<<1, 1, 0, s>>>(c->dt, c->time);
    c->launches++;
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? IBM_OK : cfail(e);
}

extern "C" ibm_status ibm_case3d_get(ibm_case3d *c, int what, void *dst, size_t bytes, int dst_on_device) {
  if (!c || !dst) return ibm__noalloc_fail(IBM_EINVAL, "ibm_case3d_get: NULL argument");
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cfail(e);
  const Grid3 &g = c->g;
  const long long nn = (long long)g.nx * g.ny * g.nz;
  const int total = c->counts[0] + c->counts[1] + c->counts[2] + c->counts[3];
  const cudaMemcpyKind kd = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  switch (what) {
    case IBM_3D_TAGS:
      if (bytes < (size_t)nn) return ibm__noalloc_fail(IBM_EINVAL, "ibm_case3d_get: dst too small");
      e = cudaMemcpy(dst, c->tags, (size_t)nn, kd);
      break;
    case IBM_3D_COUNTS:
      if (bytes < sizeof(c->counts)) return ibm__noalloc_fail(IBM_EINVAL, "ibm_case3d_get: dst too small");
      e = cudaMemcpy(dst, c->counts, sizeof(c->counts), dst_on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost);
      break;
    case IBM_3D_STENCILS:
      if (bytes < (size_t)total * sizeof(ibm_stencil3d)) return ibm__noalloc_fail(IBM_EINVAL, "ibm_case3d_get: dst too small");
      if (total) e = cudaMemcpy(dst, c->st, (size_t)total * sizeof(ibm_stencil3d), kd);
      break;
    case IBM_3D_TIME:
      if (bytes < 2 * sizeof(double)) return ibm__noalloc_fail(IBM_EINVAL, "ibm_case3d_get: dst too small");
      e = cudaMemcpy(dst, c->time, 2 * sizeof(double), kd);
      break;
    case IBM_3D_STATE: {
      if (bytes < (size_t)5 * nn * sizeof(double)) return ibm__noalloc_fail(IBM_EINVAL, "ibm_case3d_get: dst too small");
      // interior rows of every variable: one strided 3-D copy per variable
      for (int v = 0; v < 5 && e == cudaSuccess; v++) {
        cudaMemcpy3DParms prm = {};
        prm.srcPtr = make_cudaPitchedPtr(c->A.v[v], (size_t)g.W * sizeof(double), g.W, g.H);
        prm.srcPos = make_cudaPos(NG * sizeof(double), NG, NG);
        prm.dstPtr = make_cudaPitchedPtr((double *)dst + (size_t)v * nn, (size_t)g.nx * sizeof(double), g.nx, g.ny);
        prm.dstPos = make_cudaPos(0, 0, 0);
        prm.extent = make_cudaExtent((size_t)g.nx * sizeof(double), g.ny, g.nz);
        prm.kind = kd;
        e = cudaMemcpy3D(&prm);
      }
      break;
    }
    default:
      return ibm__noalloc_fail(IBM_EINVAL, "ibm_case3d_get: unknown quantity");
  }
  return e == cudaSuccess ? IBM_OK : cfail(e);
}

extern "C" ibm_status ibm_case3d_set_state(ibm_case3d *c, const void *src, size_t bytes, int src_on_device) {
  if (!c || !src) return ibm__noalloc_fail(IBM_EINVAL, "ibm_case3d_set_state: NULL argument");
  const Grid3 &g = c->g;
  const long long nn = (long long)g.nx * g.ny * g.nz;
  if (bytes < (size_t)5 * nn * sizeof(double)) return ibm__noalloc_fail(IBM_EINVAL, "ibm_case3d_set_state: src too small");
  cudaError_t e = cudaSuccess;
  for (int v = 0; v < 5 && e == cudaSuccess; v++) {
    cudaMemcpy3DParms prm = {};
    prm.srcPtr = make_cudaPitchedPtr((void *)((const double *)src + (size_t)v * nn), (size_t)g.nx * sizeof(double), g.nx, g.ny);
    prm.srcPos = make_cudaPos(0, 0, 0);
    prm.dstPtr = make_cudaPitchedPtr(c->A.v[v], (size_t)g.W * sizeof(double), g.W, g.H);
    prm.dstPos = make_cudaPos(NG * sizeof(double), NG, NG);
    prm.extent = make_cudaExtent((size_t)g.nx * sizeof(double), g.ny, g.nz);
    prm.kind = src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    e = cudaMemcpy3DAsync(&prm, c->stream);
  }
  if (e == cudaSuccess && c->precision == IBM_PREC_FP32_BULK) {
    k3_mirror32<<<cells(g.W, g.H, g.D), CB, 0, c->stream>>>(g, c->ph, c->A, c->mirror);
    c->launches++;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && !src_on_device) e = cudaStreamSynchronize(c->stream);
  return e == cudaSuccess ? IBM_OK : cfail(e);
}

extern "C" ibm_status ibm_case3d_forces(ibm_case3d *c, double out[6]) {
  if (!c || !out) return ibm__noalloc_fail(IBM_EINVAL, "ibm_case3d_forces: NULL argument");
  double F[3] = {0.0, 0.0, 0.0};
  cudaError_t e = cudaSuccess;
  if (c->ntri > 0) {
    k3_surface_force<<<nblk(c->ntri), TB, 0, c->stream>>>(c->g, c->ph, c->A, c->sst, c->tri + (size_t)6 * c->ntri,
                                                          c->ntri, c->fbuf);
    k3_force_sum<<<1, TB, 0, c->stream>>>(c->fbuf, c->ntri, c->fbuf + (size_t)3 * c->ntri);
    c->launches += 2;
    e = cudaMemcpyAsync(F, c->fbuf + (size_t)3 * c->ntri, sizeof(F), cudaMemcpyDeviceToHost, c->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cfail(e);
  const double qref = 0.5 * c->ref_area;  // 1/2 rho_inf U_ref^2 A_ref with rho_inf = U_ref = 1
  for (int a = 0; a < 3; a++) {
    out[a] = F[a] / qref;
    out[3 + a] = F[a];
  }
  return IBM_OK;
}

extern "C" int64_t ibm_case3d_launch_count(const ibm_case3d *c) { return c ? c->launches : 0; }
