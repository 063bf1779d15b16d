// Dual-time pseudo-stage update of one fluid cell in FP32-bulk form (FP64
// arithmetic), included by stage32.cuh ahead of the per-tile code.
#pragma once

#include "ibm_internal.cuh"

namespace ibm {

// ---------------------------------------------------------------------------
// Dual time in FP32-bulk form (Sec. 2).  The residual of a pseudo stage is the
// FP32 perturbation residual above (preconditioned LDFSS faces); the
// point-implicit update of each fluid cell runs in FP64:
//   [T Gamma / dtau + a T dW/dQ] dQ = -(R' + BDF'),   a = 3/(2 dt) or 1/dt,
// in perturbation variables W' = T W (T subtracts H_inf times the mass row
// from the energy row), so the energy rows of the Weiss-Smith matrices carry
// H - H_inf instead of H and never cancel against H_inf; R' = -L is the FP32
// residual, BDF' is formed from the FP64 iterate and the time levels' part
// fixed for the physical step (formed once per step), the 4x4
// system is solved in FP64 through its structure (solve_precond; the
// reciprocal of its FP32 pseudo-time step coefficient in FP32),
// Q' = (p', u, v, T') is updated and combined with the sub-iteration's start
// as SSP-RK3 stage, and the new iterate is stored in FP64 with its FP32
// mirror.
// ---------------------------------------------------------------------------
struct DualPtrs {
  const double *In64;  // FP64 iterate the stage starts from (perturbation)
  double *Out64;       // FP64 iterate it produces
  const double *G;     // the physical step's constant part of the BDF term: (W^{n-1} - 4 W^n) / (2 dt), or
                       // -W^n / dt on the first step (perturbation)
  double *Q0;          // (p', u, v, T') of the sub-iteration's start: written by stage 1, read by 2 and 3
};

// IEEE 754 binary32 <-> binary64 conversions done on the integer bits, off the
// FP64 pipe (which bounds the pseudo stage).  f32_to_f64 is exact for every
// normal and zero value (the FP32 arithmetic here flushes subnormals to
// zero); f64_to_f32 rounds to nearest, ties to even, for results in the
// normal FP32 range and leaves anything else to the hardware conversion.
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned int b = __float_as_uint(f), e = (b >> 23) & 0xffu;
  if (e == 0xffu) return (double)f;  // infinity or NaN
  const unsigned int hi = (b & 0x80000000u) | (e ? ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3) : 0u);
  return __hiloint2double((int)hi, (int)(e ? b << 29 : 0u));
}
__device__ __forceinline__ float f64_to_f32(double d) {
  const unsigned int hi = (unsigned int)__double2hiint(d), lo = (unsigned int)__double2loint(d);
  const unsigned int e = (hi >> 20) & 0x7ffu;
  if (e - 897u >= 254u) return (float)d;  // outside the normal FP32 exponent range: hardware conversion
  unsigned int f = (hi & 0x80000000u) | ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  const unsigned int rest = lo & 0x1fffffffu;  // the 29 dropped mantissa bits
  f += (rest > 0x10000000u) | ((rest == 0x10000000u) & (f & 1u));
  return __uint_as_float(f);
}

// FP64 perturbation conserved -> (p', u, v, T'); ir receives 1 / rho.  Reciprocals here are the
// round-to-nearest FP64 reciprocal (the iterate's conversions stay exact to FP64 rounding).
__device__ __forceinline__ void pert_prim64(const Consts &k, double dr, double dmx, double dmy, double W,
                                            double q[4], double &ir) {
  const double r = 1.0 + dr;
  ir = __drcp_rn(r);
  const double u = (k.uinf[0] + dmx) * ir, v = (k.uinf[1] + dmy) * ir;
  const double du = (dmx - dr * k.uinf[0]) * ir, dv = (dmy - dr * k.uinf[1]) * ir;
  const double dq = du * (u + k.uinf[0]) + dv * (v + k.uinf[1]);
  const double ke = 0.5 * (dr * (u * u + v * v) + dq);
  const double pp = (k.gamma - 1.0) * (W + k.Hinf * dr - ke);
  q[0] = pp;
  q[1] = u;
  q[2] = v;
  q[3] = (pp - k.R * dr) * ir * k.iR;
}

// (p', u, v, T') -> FP64 perturbation conserved
__device__ __forceinline__ void prim_pert64(const Consts &k, const double q[4], double w[4]) {
  const double pp = q[0], u = q[1], v = q[2], Tp = q[3];
  const double dr = (pp - k.R * Tp) * k.iR * __drcp_rn(1.0 + Tp);
  const double dq = (u - k.uinf[0]) * (u + k.uinf[0]) + (v - k.uinf[1]) * (v + k.uinf[1]);
  const double ke = 0.5 * (dr * (u * u + v * v) + dq);
  w[0] = dr;
  w[1] = dr * u + (u - k.uinf[0]);
  w[2] = dr * v + (v - k.uinf[1]);
  w[3] = pp * k.ig1 + ke - k.Hinf * dr;
}

// Exact solution of the point-implicit system in perturbation rows.  With
// s = 1/dtau + a the operator is s times the Weiss-Smith matrix whose first
// column parameter is tau = (theta_G/dtau + a theta_J) / s (the other columns
// are shared by Gamma and dW/dQ), so the momentum rows give du, dv directly
// (after subtracting u, v times the first row) and the first and energy rows
// leave a 2x2 system in dp, dT:
//   tau dp + rho_T dT = S0/s,   -dp + rho cp dT = (S3 - dH S0)/s - rho (u du + v dv).
// is = 1/s, ir = 1/rho.  1/s scales the whole update (a pseudo-time step
// size: it sets the path in pseudo time, not the fixed point, which the FP64
// right-hand side S fixes) and is taken in FP32 like s itself.  The pivot
// tau rho cp + rho_T is inverted in FP64: dp = rho cp dT - X is a small
// difference of two terms of size X, so a relative error in 1/pivot would
// reach dp multiplied by X / dp.
__device__ __forceinline__ void solve_precond(double is, double tau, double r, double ir, double u, double v,
                                              double rT, double cpv, double dH, const double S[4], double dQ[4]) {
  const double irs = is * ir;
  const double du = (S[1] - u * S[0]) * irs;
  const double dv = (S[2] - v * S[0]) * irs;
  const double X = (S[3] - dH * S[0]) * is - r * (u * du + v * dv);
  const double Y = S[0] * is;
  const double dT = (Y + tau * X) * __drcp_rn(tau * r * cpv + rT);
  dQ[0] = r * cpv * dT - X;
  dQ[1] = du;
  dQ[2] = dv;
  dQ[3] = dT;
}

// pseudo stage STAGE of one fluid cell (id: state index); L = FP32 residual
template <int STAGE>
__device__ __forceinline__ void dual_update_cell(const Consts &k, const PertConsts &c, long long id, long long P,
                                                 const float L[4], const DualPtrs &dp,
                                                 float *Out32, bool bdf2) {
  const double idt = k.idt_phys;
  const double aw = bdf2 ? 1.5 * idt : idt;  // coefficient of the iterate in the BDF term
  double W[4], S[4], Qk[4], ir;
  for (int v = 0; v < 4; v++) W[v] = dp.In64[id + v * P];
  pert_prim64(k, W[0], W[1], W[2], W[3], Qk, ir);
  for (int v = 0; v < 4; v++) {
    const double tdt = aw * W[v] + dp.G[id + v * P];  // BDF2 (3 W - 4 W^n + W^{n-1}) / (2 dt), BDF1 (W - W^n) / dt
    S[v] = f32_to_f64(L[v]) - tdt;                     // -(R' + BDF') with R' = -L
  }
  // pseudo-time coefficients (local dtau, preconditioning parameter) in FP32: they set the pseudo-time path,
  // not the fixed point R' + BDF' = 0
  const double r = 1.0 + W[0], u = Qk[1], v = Qk[2];
  const float rf = f64_to_f32(r), irf = 1.f / rf, uf = f64_to_f32(u), vf = f64_to_f32(v);
  const float Tf = 1.f + f64_to_f32(Qk[3]), iTf = 1.f / Tf;
  const float csf = sqrtf(c.gamma * (c.R + f64_to_f32(Qk[0])) * irf), icsf = 1.f / csf;
  const float Vm = sqrtf(uf * uf + vf * vf);
  float Ur = fmaxf(fmaxf(Vm, 1.f), c.mu * irf / c.dmin);
  Ur = fminf(Ur, csf);
  const float mr2 = (Ur * icsf) * (Ur * icsf);
  const float up = 0.5f * Vm * (1.f + mr2);
  const float om = 1.f - mr2;
  const float cp_ = 0.5f * sqrtf(om * om * Vm * Vm + 4.f * Ur * Ur);
  const float lam = (up + cp_) * (c.idx + c.idy) + c.vis * irf;
  const float idtau = lam / c.cfl_tau;
  const float af = bdf2 ? 1.5f * c.idt_phys : c.idt_phys;
  const float thG = 1.f / (Ur * Ur) + iTf / c.cp, thJ = iTf / c.R;
  const float sf = idtau + af;
  const float tau = (thG * idtau + af * thJ) / sf;
  const double dH = k.cp * Qk[3] + 0.5 * ((u - k.uinf[0]) * (u + k.uinf[0]) + (v - k.uinf[1]) * (v + k.uinf[1]));
  double dQ[4];
  solve_precond(f32_to_f64(1.f / sf), f32_to_f64(tau), r, ir, u, v, -f32_to_f64(rf * iTf), k.cp, dH, S, dQ);
  double Q0[4], Qn[4], Wo[4];
  if (STAGE == 1) {  // the stage starts from the sub-iteration's start: keep its primitives for stages 2 and 3
    for (int q = 0; q < 4; q++) dp.Q0[id + q * P] = Qk[q];
  } else {
    for (int q = 0; q < 4; q++) Q0[q] = dp.Q0[id + q * P];
  }
  for (int q = 0; q < 4; q++) {
    const double e = Qk[q] + dQ[q];
    Qn[q] = STAGE == 1 ? e : (STAGE == 2 ? 0.75 * Q0[q] + 0.25 * e : (1.0 / 3.0) * Q0[q] + (2.0 / 3.0) * e);
  }
  prim_pert64(k, Qn, Wo);
  for (int q = 0; q < 4; q++) {
    dp.Out64[id + q * P] = Wo[q];
    Out32[id + q * P] = f64_to_f32(Wo[q]);
  }
}

}  // namespace ibm
