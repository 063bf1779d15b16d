// FP64 flow kernels: time step, IB / ghost reconstruction and the fused
// residual + SSP-RK3 stage update (domain halos are applied while the stage
// kernel loads its tile).
//
// State layout: structure of arrays, four conserved planes (rho, rho u,
// rho v, rho E), each (ny + 6) rows of `pitch` doubles; cell (i, j) of the
// interior sits at (j + 3) * pitch + (i + 3).  Rows are padded to a multiple
// of 32 elements so every row starts 256-byte aligned.
#include "ibm_internal.cuh"

namespace ibm {

// ---------------------------------------------------------------------------
// Time step from the CFL rule over fluid cells:
//   dt = CFL / max[(|u|+c)/dx + (|v|+c)/dy + 2 gamma mu/(Pr rho)(1/dx^2+1/dy^2)].
// Positive doubles order like their bit patterns, so the maximum is an
// integer atomicMax (order-independent, exact); the last block to finish
// turns it into dt.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_dt(Consts k, const double *__restrict__ A,
                                            const uint8_t *__restrict__ tag, DevState *ds) {
  const int ncell = k.nx * k.ny;
  double lmax = 0.0;
  const double vis = (2.0 * k.gamma * k.mu / k.prandtl) * (1.0 / (k.dx * k.dx) + 1.0 / (k.dy * k.dy));
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < ncell; n += gridDim.x * blockDim.x) {
    if (tag[n] != FLUID && !(k.ib_advance && tag[n] == IB)) continue;
    long long id = cidx(k, n % k.nx, n / k.nx);
    double r = A[id], u = A[id + k.plane] / r, v = A[id + 2 * k.plane] / r;
    double p = (k.gamma - 1.0) * (A[id + 3 * k.plane] - 0.5 * r * (u * u + v * v));
    double c = sqrt(k.gamma * p / r);
    double lam = (fabs(u) + c) / k.dx + (fabs(v) + c) / k.dy + vis / r;
    lmax = fmax(lmax, lam);
  }
  for (int off = 16; off > 0; off >>= 1) lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, off));
  __shared__ double wm[8];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = lmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = wm[0];
    for (int w = 1; w < 8; w++) m = fmax(m, wm[w]);
    atomicMax(&ds->lmax_bits, (unsigned long long)__double_as_longlong(m));
    finish_cfl(k, ds, gridDim.x * gridDim.y);
  }
}

void launch_dt(const Consts &k, const double *A, const uint8_t *tag, DevState *ds, cudaStream_t s, int *nlaunch) {
  if (k.dt_fixed > 0.0) return;  // ds->dt was set at creation
  int ncell = k.nx * k.ny;
  int blocks = min((ncell + 255) / 256, 152 * 8);
  k_dt<<<blocks, 256, 0, s>>>(k, A, tag, ds);
  *nlaunch += 1;
}

// ---------------------------------------------------------------------------
// Sec. 4.4-4.6, Sec. 5: rebuild IB nodes (pass 0) or ghost nodes (pass 1)
// from their stencils.  Primitives p, u, v, T are interpolated at the probe
// / image point; velocity is Dirichlet (Eq. 4), linear along the normal
// through the wall velocity at P'; pressure is Neumann with
// dp/dn = -rho n.a_wall (Eq. 5-6), plus, for a body moving faster than the
// free-stream sound speed, the centripetal term rho u_t^2 kappa of the normal
// momentum balance (Eq. 7, in the sign convention of Eq. 6; u_t is the
// velocity tangential to the wall relative to it at the probe, kappa the
// signed curvature at P'); temperature is adiabatic (Eq. 8), which makes the
// pressure condition a linear ODE in p along the normal, integrated exactly.
// One thread per list entry; in place on the stage array.
// ---------------------------------------------------------------------------
// A state written by the caller ([4][ny][nx] absolute conserved, contiguous, already on the device) into the
// case's padded layout: FP64 as given, or -- FP32-bulk, M != null -- as the perturbation from the free stream
// (dU = U - U_inf, the energy row less H_inf d rho) with its FP32 mirror.  One thread per cell.
__global__ void k_set_state(Consts k, const double *__restrict__ U, double *__restrict__ A, float *__restrict__ M) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long ncell = (long long)k.nx * k.ny;
  if (n >= ncell) return;
  const long long id = cidx(k, (int)(n % k.nx), (int)(n / k.nx)), P = k.plane;
  double u0 = U[n], u1 = U[n + ncell], u2 = U[n + 2 * ncell], u3 = U[n + 3 * ncell];
  if (M) {
    const double d = u0 - 1.0;
    u0 = d;
    u1 = u1 - k.Uinf[1];
    u2 = u2 - k.Uinf[2];
    u3 = (u3 - k.Uinf[3]) - k.Hinf * d;
    M[id] = (float)u0;
    M[id + P] = (float)u1;
    M[id + 2 * P] = (float)u2;
    M[id + 3 * P] = (float)u3;
  }
  A[id] = u0;
  A[id + P] = u1;
  A[id + 2 * P] = u2;
  A[id + 3 * P] = u3;
}

void launch_set_state(const Consts &k, const double *U, double *A, float *M, cudaStream_t s) {
  const long long ncell = (long long)k.nx * k.ny;
  k_set_state<<<(unsigned)((ncell + 255) / 256), 256, 0, s>>>(k, U, A, M);
}

// (p, u, v, T) interpolated at a probe from the valid corners of its square
__device__ __forceinline__ void probe_f64(const Consts &k, const double *U, int i0, int j0, int mask,
                                          const double w[4], double qp[4]) {
  for (int q = 0; q < 4; q++) qp[q] = 0.0;
  for (int q = 0; q < 4; q++) {
    if (!(mask >> q & 1)) continue;
    long long id = cidx(k, i0 + (q & 1), j0 + (q >> 1));
    double r = U[id], u = U[id + k.plane] / r, v = U[id + 2 * k.plane] / r;
    double p = (k.gamma - 1.0) * (U[id + 3 * k.plane] - 0.5 * r * (u * u + v * v));
    qp[0] += w[q] * p;
    qp[1] += w[q] * u;
    qp[2] += w[q] * v;
    qp[3] += w[q] * (p / (r * k.R));
  }
}

__device__ __forceinline__ void recon_one_f64(const Consts &k, double *U, const ibm_stencil &s, const double Vb[2],
                                              const double Ab[2], bool sup, double t) {
  if (s.mask == 0) return;
  double V[2], Acc[2];
  wall_kin(k, t, s.bx, s.by, Vb, Ab, V, Acc);  // the wall's motion at P'
  double qp[4];
  probe_f64(k, U, s.i0, s.j0, s.mask, s.w, qp);
  // dp/dn = rho G (Eq. 5-7)
  double G = -(s.nx * Acc[0] + s.ny * Acc[1]);
  if (sup) {
    const double ut = -(qp[1] - V[0]) * s.ny + (qp[2] - V[1]) * s.nx;
    G = G + ut * ut * s.curv;
  }
  double p, u, v, T;
  if (k.quad && s.maskb != 0) {
    // quadratic form (Sec. 4.5, Sec. 5): quadratics in the distance s along the normal through the wall
    // condition (s = 0) and the probes at s1, s2, evaluated at the node s_n -- Lagrange for the Dirichlet
    // velocity, a + b s + c s^2 with the wall slope b given for T (0) and p (rho G, the first probe's density)
    double qb[4];
    probe_f64(k, U, s.i0b, s.j0b, s.maskb, s.wb, qb);
    const double s1 = s.xi_probe, s2 = s.xi_probe2, sn = s.xi_node;
    const double L1 = sn * (sn - s2) / (s1 * (s1 - s2)), L2 = sn * (sn - s1) / (s2 * (s2 - s1));
    const double m = (sn * sn - s1 * s1) / (s2 * s2 - s1 * s1);
    const double b = qp[0] / (k.R * qp[3]) * G;
    u = V[0] + (qp[1] - V[0]) * L1 + (qb[1] - V[0]) * L2;
    v = V[1] + (qp[2] - V[1]) * L1 + (qb[2] - V[1]) * L2;
    T = qp[3] + (qb[3] - qp[3]) * m;
    p = qp[0] + (qb[0] - qp[0]) * m + b * ((sn - s1) - (s2 - s1) * m);
  } else {
    // linear form: rho = p / (R T) and T fixed along the normal (Eq. 8), integrated exactly from the probe to
    // the node, p = p_probe exp(-(xi_p - xi_n) G / (R T)), positive however coarse the grid
    const double ratio = s.xi_node / s.xi_probe;
    p = qp[0] * exp(-(s.xi_probe - s.xi_node) * G / (k.R * qp[3]));
    u = V[0] + (qp[1] - V[0]) * ratio;
    v = V[1] + (qp[2] - V[1]) * ratio;
    T = qp[3];
  }
  const double r = p / (k.R * T);
  const long long id = cidx(k, s.cell % k.nx, s.cell / k.nx);
  U[id] = r;
  U[id + k.plane] = r * u;
  U[id + 2 * k.plane] = r * v;
  U[id + 3 * k.plane] = p / (k.gamma - 1.0) + 0.5 * r * (u * u + v * v);
}

// one block: all IB nodes, a barrier, then all ghost nodes
__global__ void __launch_bounds__(1024) k_recon1_f64(Consts k, double *U, const ibm_stencil *__restrict__ st,
                                                     int cap, const DevState *__restrict__ ds, int stage) {
  double X[2], V[2], Acc[2];
  const double ts = stage_time(ds, stage);
  body_motion(k, ds, ts, X, V, Acc);
  const bool sup = supersonic_motion(k, V);
  const int nib = min(ds->offset[1], cap), tot = min(ds->offset[4], cap);
  if (!k.ib_advance)  // IB nodes rebuilt (else advanced by the flux update)
    for (int e = threadIdx.x; e < nib; e += blockDim.x) recon_one_f64(k, U, st[e], V, Acc, sup, ts);
  __syncthreads();
  for (int e = nib + threadIdx.x; e < tot; e += blockDim.x) recon_one_f64(k, U, st[e], V, Acc, sup, ts);
}

// many blocks, one pass (0: IB nodes, 1: ghost nodes) per launch
__global__ void __launch_bounds__(128) k_recon_f64(Consts k, double *U, const ibm_stencil *__restrict__ st,
                                                   int cap, const DevState *__restrict__ ds, int stage, int pass) {
  const int lo = pass == 0 ? 0 : ds->offset[1];
  const int hi = min(pass == 0 ? ds->offset[1] : ds->offset[4], cap);
  const int e = lo + blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= hi) return;
  double X[2], V[2], Acc[2];
  const double ts = stage_time(ds, stage);
  body_motion(k, ds, ts, X, V, Acc);
  recon_one_f64(k, U, st[e], V, Acc, supersonic_motion(k, V), ts);
}

void launch_recon_f64(const Consts &k, double *U, const ibm_stencil *st, int cap, const DevState *ds, int stage,
                      cudaStream_t s, int *nlaunch) {
  if (cap <= 0) return;
  if (cap <= RECON_ONE_BLOCK_MAX) {
    k_recon1_f64<<<1, 1024, 0, s>>>(k, U, st, cap, ds, stage);
    *nlaunch += 1;
    return;
  }
  int blocks = (cap + 127) / 128;
  if (!k.ib_advance) {  // IB nodes rebuilt (else advanced by the flux update)
    k_recon_f64<<<blocks, 128, 0, s>>>(k, U, st, cap, ds, stage, 0);
    *nlaunch += 1;
  }
  k_recon_f64<<<blocks, 128, 0, s>>>(k, U, st, cap, ds, stage, 1);
  *nlaunch += 1;
}

// ---------------------------------------------------------------------------
// Sec. 2: fifth-order WENO (Jiang-Shu smoothness indicators, linear weights
// 1/10, 6/10, 3/10, eps = 1e-6); value at the face right of f2.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R weno5(R f0, R f1, R f2, R f3, R f4) {
  const R eps = R(1e-6);
  R a = f0 - R(2) * f1 + f2, b = f0 - R(4) * f1 + R(3) * f2;
  R b0 = R(13.0 / 12.0) * a * a + R(0.25) * b * b;
  a = f1 - R(2) * f2 + f3;
  b = f1 - f3;
  R b1 = R(13.0 / 12.0) * a * a + R(0.25) * b * b;
  a = f2 - R(2) * f3 + f4;
  b = R(3) * f2 - R(4) * f3 + f4;
  R b2 = R(13.0 / 12.0) * a * a + R(0.25) * b * b;
  R q0 = (R(2) * f0 - R(7) * f1 + R(11) * f2) * R(1.0 / 6.0);
  R q1 = (-f1 + R(5) * f2 + R(2) * f3) * R(1.0 / 6.0);
  R q2 = (R(2) * f2 + R(5) * f3 - f4) * R(1.0 / 6.0);
  R e0 = eps + b0, e1 = eps + b1, e2 = eps + b2;
  // a_k = d_k / e_k^2, normalised; one division for all three weights
  R e01 = e0 * e1, e12 = e1 * e2, e02 = e0 * e2;
  R a0 = R(0.1) * e12 * e12, a1 = R(0.6) * e02 * e02, a2 = R(0.3) * e01 * e01;
  return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
}

// Sec. 2, the second-order TVD scheme: MUSCL with the minmod limiter; value at the face right of f1
template <typename R>
__device__ __forceinline__ R tvd2(R f0, R f1, R f2) {
  const R a = f1 - f0, b = f2 - f1;
  R m = R(0);
  if (a > R(0) && b > R(0)) m = a < b ? a : b;
  else if (a < R(0) && b < R(0)) m = a > b ? a : b;
  return f1 + R(0.5) * m;
}

// ---------------------------------------------------------------------------
// Sec. 2: LDFSS(0) face flux (plain, Mr^2 = 1: explicit time stepping does
// not precondition the dissipation).  States (rho, u, v, p); normal along
// the first velocity component un, tangential ut.  F = (mass, normal
// momentum, tangential momentum, energy).
// ---------------------------------------------------------------------------
template <bool PRE>
__device__ __forceinline__ void ldfss_f64(double rL, double unL, double utL, double pL, double rR, double unR,
                                          double utR, double pR, double gamma, double mr2, double F[4]) {
  const double gg = gamma / (gamma - 1.0);
  const double cL = sqrt(gamma * pL / rL), cR = sqrt(gamma * pR / rR);
  const double HL = gg * pL / rL + 0.5 * (unL * unL + utL * utL);
  const double HR = gg * pR / rR + 0.5 * (unR * unR + utR * utR);
  const double cb = 0.5 * (cL + cR);
  double cs = cb;
  if (PRE) {  // low-Mach numerical sound speed c' = 1/2 sqrt((1-Mr^2)^2 un^2 + 4 Mr^2 c^2)
    const double ub = 0.5 * (unL + unR), om = 1.0 - mr2;
    cs = 0.5 * sqrt(om * om * ub * ub + 4.0 * mr2 * cb * cb);
  }
  const double ics = 1.0 / cs;
  const double ML = unL * ics, MR = unR * ics;
  const double aL = ML >= 0.0 ? 1.0 : 0.0;
  const double aR = MR >= 0.0 ? 0.0 : 1.0;
  const double tL = 1.0 - floor(fabs(ML)), tR = 1.0 - floor(fabs(MR));
  const double bL = -fmax(tL, 0.0), bR = -fmax(tR, 0.0);
  const double MpL = 0.25 * (ML + 1.0) * (ML + 1.0);
  const double MmR = -0.25 * (MR - 1.0) * (MR - 1.0);
  const double CVL = aL * (1.0 + bL) * ML - bL * MpL;
  const double CVR = aR * (1.0 + bR) * MR - bR * MmR;
  const double sq = sqrt(0.5 * (ML * ML + MR * MR)) - 1.0;
  const double Mh = 0.25 * bL * bR * sq * sq;
  const double dp = pL - pR, adp = fabs(dp);
  const double ic2 = 0.5 * ics * ics;
  const double MhP = Mh * (1.0 - (dp + adp) * ic2 / rL);
  const double MhM = Mh * (1.0 - (adp - dp) * ic2 / rR);
  const double Cp = CVL - MhP, Cm = CVR + MhM;
  double DL, DR;
  if (PRE && mr2 < 1.0) {  // pressure split with the physical Mach numbers (its dissipation scaled below)
    const double ic = 1.0 / cb;
    const double mL = unL * ic, mR = unR * ic;
    const double paL = mL >= 0.0 ? 1.0 : 0.0, paR = mR >= 0.0 ? 0.0 : 1.0;
    const double pbL = -fmax(1.0 - floor(fabs(mL)), 0.0), pbR = -fmax(1.0 - floor(fabs(mR)), 0.0);
    const double PpL = 0.25 * (mL + 1.0) * (mL + 1.0) * (2.0 - mL);
    const double PmR = 0.25 * (mR - 1.0) * (mR - 1.0) * (2.0 + mR);
    DL = paL * (1.0 + pbL) - pbL * PpL;
    DR = paR * (1.0 + pbR) - pbR * PmR;
  } else {
    const double PpL = MpL * (2.0 - ML);
    const double PmR = -MmR * (2.0 + MR);
    DL = aL * (1.0 + bL) - bL * PpL;
    DR = aR * (1.0 + bR) - bR * PmR;
  }
  const double mL = rL * cs * Cp, mR = rR * cs * Cm;
  double ph = DL * pL + DR * pR;
  if (PRE && mr2 < 1.0) {
    // low-Mach scaling: the split's departure from the face mean (its rho c du dissipation) times c'/c
    const double fa = cs / cb;
    ph = 0.5 * (pL + pR) + fa * ((DL - 0.5) * pL + (DR - 0.5) * pR);
  }
  F[0] = mL + mR;
  F[1] = mL * unL + mR * unR + ph;
  F[2] = mL * utL + mR * utR;
  F[3] = mL * HL + mR * HR;
}

// ---------------------------------------------------------------------------
// Fused residual + stage update, FP64.  One 16x16 tile of cells per block:
// the tile and its 3-cell halo are loaded once, converted to primitives in
// shared memory; every x- and y-face of the tile is computed once (WENO5 +
// LDFSS + central viscous flux); each fluid cell then takes the flux
// divergence and applies its SSP-RK3 stage:
//   stage 1: out = Un + dt L(in)
//   stage 2: out = 3/4 Un + 1/4 (in + dt L(in))
//   stage 3: out = 1/3 Un + 2/3 (in + dt L(in))
// Tiles without a fluid cell exit at once.
// ---------------------------------------------------------------------------
constexpr int TX = 16, TY = 16, HX = TX + 2 * NG, HY = TY + 2 * NG;

// Low-Mach preconditioning parameter at a face (dual time): reference velocity
// Ur = min(c, max(|V|, U_ref, nu/dn)) from face-averaged c, |V|, rho;
// returns Mr^2 = (Ur/c)^2.  States (rho, u, v, p).
__device__ __forceinline__ double face_mr2(const Consts &k, const double qL[4], const double qR[4], double dn) {
  const double cb = 0.5 * (sqrt(k.gamma * qL[3] / qL[0]) + sqrt(k.gamma * qR[3] / qR[0]));
  const double ub = 0.5 * (qL[1] + qR[1]), vb = 0.5 * (qL[2] + qR[2]);
  const double Vm = sqrt(ub * ub + vb * vb);
  const double rb = 0.5 * (qL[0] + qR[0]);
  double Ur = fmax(fmax(Vm, 1.0), k.mu / rb / dn);
  Ur = fmin(Ur, cb);
  const double m = (Ur / cb) * (Ur / cb);
  return fmin(m, 1.0);
}

// Weiss-Smith matrix in Q = (p, u, v, T) with first-column parameter theta:
// Gamma (theta = 1/Ur^2 - rT/(r cp)) or dW/dQ (theta = 1/(R T)); row major
__device__ __forceinline__ void wq_matrix(double theta, double p, double u, double v, double T, double r, double cpv,
                                          double M[16]) {
  const double rT = -r / T;
  const double H = cpv * T + 0.5 * (u * u + v * v);
  M[0] = theta;           M[1] = 0.0;    M[2] = 0.0;    M[3] = rT;
  M[4] = theta * u;       M[5] = r;      M[6] = 0.0;    M[7] = rT * u;
  M[8] = theta * v;       M[9] = 0.0;    M[10] = r;     M[11] = rT * v;
  M[12] = theta * H - 1.0; M[13] = r * u; M[14] = r * v; M[15] = rT * H + r * cpv;
  (void)p;
}

// Gaussian elimination with partial pivoting; false if singular
__device__ __forceinline__ bool solve4(double A[16], double b[4], double x[4]) {
#pragma unroll
  for (int col = 0; col < 4; col++) {
    int piv = col;
#pragma unroll
    for (int i = col + 1; i < 4; i++)
      if (fabs(A[4 * i + col]) > fabs(A[4 * piv + col])) piv = i;
    if (A[4 * piv + col] == 0.0) return false;
    if (piv != col) {
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const double t = A[4 * col + j];
        A[4 * col + j] = A[4 * piv + j];
        A[4 * piv + j] = t;
      }
      const double t = b[col];
      b[col] = b[piv];
      b[piv] = t;
    }
#pragma unroll
    for (int i = col + 1; i < 4; i++) {
      const double f = A[4 * i + col] / A[4 * col + col];
#pragma unroll
      for (int j = col; j < 4; j++) A[4 * i + j] -= f * A[4 * col + j];
      b[i] -= f * b[col];
    }
  }
#pragma unroll
  for (int i = 3; i >= 0; i--) {
    double s = b[i];
#pragma unroll
    for (int j = i + 1; j < 4; j++) s -= A[4 * i + j] * x[j];
    x[i] = s / A[4 * i + i];
  }
  return true;
}

template <int STAGE, bool DUAL>
__global__ void __launch_bounds__(256) k_stage_f64(Consts k, const double *Un, const double *__restrict__ In,
                                                   double *Out, const double *__restrict__ Wn,
                                                   const double *__restrict__ Wm, const uint8_t *__restrict__ tag,
                                                   DevState *ds) {
  __shared__ double sq[4][HY][HX];  // rho, u, v, p
  __shared__ double sT[HY][HX];     // temperature
  __shared__ double sfx[4][TY][TX + 1];
  __shared__ double sfy[4][TY + 1][TX];
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int ci = i0 + tx, cj = j0 + ty;
  const bool inside = ci < k.nx && cj < k.ny;
  // cells the flux update advances: fluid cells, and IB nodes when the ghost layers alone impose the wall
  const bool fluid = inside && (tag[cj * k.nx + ci] == FLUID || (k.ib_advance && tag[cj * k.nx + ci] == IB));
  const double dt = ds->dt;
  if (!DUAL && STAGE == 3 && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
    // end of the step (no other kernel of this stage reads t)
    ds->t = ds->t + dt;
    ds->steps += 1;
  }
  if (!__syncthreads_or(fluid)) return;

  const long long P = k.plane;
  const double g1 = k.gamma - 1.0;
  for (int m = threadIdx.x; m < HX * HY; m += 256) {
    const int a = m % HX, b = m / HX;
    int gi = i0 - NG + a, gj = j0 - NG + b;
    double U0, U1, U2, U3;
    if (halo_map(k, gi, gj)) {
      const long long id = cidx(k, gi, gj);
      U0 = In[id];
      U1 = In[id + P];
      U2 = In[id + 2 * P];
      U3 = In[id + 3 * P];
    } else {
      U0 = k.Uinf[0];
      U1 = k.Uinf[1];
      U2 = k.Uinf[2];
      U3 = k.Uinf[3];
    }
    const double r = U0;
    const double ir = 1.0 / r;
    const double u = U1 * ir, v = U2 * ir;
    const double p = g1 * (U3 - 0.5 * r * (u * u + v * v));
    sq[0][b][a] = r;
    sq[1][b][a] = u;
    sq[2][b][a] = v;
    sq[3][b][a] = p;
    sT[b][a] = p * ir / k.R;
  }
  __syncthreads();

  const double mu = k.mu, kap = k.kappa;
  const double idx = 1.0 / k.dx, idy = 1.0 / k.dy;
  // x-faces: face f sits between local columns f+2 and f+3 (global i0-1+f, i0+f)
  for (int m = threadIdx.x; m < (TX + 1) * TY; m += 256) {
    const int f = m % (TX + 1), row = m / (TX + 1);
    const int b = row + NG;
    double qL[4], qR[4];
    for (int v = 0; v < 4; v++) {
      const double *s = &sq[v][b][f];
      if (k.tvd2) {
        qL[v] = tvd2(s[1], s[2], s[3]);
        qR[v] = tvd2(s[4], s[3], s[2]);
      } else {
        qL[v] = weno5(s[0], s[1], s[2], s[3], s[4]);
        qR[v] = weno5(s[5], s[4], s[3], s[2], s[1]);
      }
    }
    if (!(qL[0] > 0.0) || !(qL[3] > 0.0) || !(qR[0] > 0.0) || !(qR[3] > 0.0)) {
      for (int v = 0; v < 4; v++) {
        qL[v] = sq[v][b][f + 2];
        qR[v] = sq[v][b][f + 3];
      }
    }
    double F[4];
    ldfss_f64<DUAL>(qL[0], qL[1], qL[2], qL[3], qR[0], qR[1], qR[2], qR[3], k.gamma,
                    DUAL ? face_mr2(k, qL, qR, k.dx) : 1.0, F);
    const int a = f + 2, a1 = f + 3;
    const double ux = (sq[1][b][a1] - sq[1][b][a]) * idx;
    const double vx = (sq[2][b][a1] - sq[2][b][a]) * idx;
    const double Tx = (sT[b][a1] - sT[b][a]) * idx;
    const double uy = (sq[1][b + 1][a] - sq[1][b - 1][a] + sq[1][b + 1][a1] - sq[1][b - 1][a1]) * (0.25 * idy);
    const double vy = (sq[2][b + 1][a] - sq[2][b - 1][a] + sq[2][b + 1][a1] - sq[2][b - 1][a1]) * (0.25 * idy);
    const double txx = mu * ((4.0 / 3.0) * ux - (2.0 / 3.0) * vy);
    const double txy = mu * (uy + vx);
    const double uf = 0.5 * (sq[1][b][a] + sq[1][b][a1]), vf = 0.5 * (sq[2][b][a] + sq[2][b][a1]);
    sfx[0][row][f] = F[0];
    sfx[1][row][f] = F[1] - txx;
    sfx[2][row][f] = F[2] - txy;
    sfx[3][row][f] = F[3] - (uf * txx + vf * txy + kap * Tx);
  }
  // y-faces: face f sits between local rows f+2 and f+3
  for (int m = threadIdx.x; m < TX * (TY + 1); m += 256) {
    const int col = m % TX, f = m / TX;
    const int a = col + NG;
    double qL[4], qR[4];
    for (int v = 0; v < 4; v++) {
      const double s0 = sq[v][f][a], s1 = sq[v][f + 1][a], s2 = sq[v][f + 2][a];
      const double s3 = sq[v][f + 3][a], s4 = sq[v][f + 4][a], s5 = sq[v][f + 5][a];
      if (k.tvd2) {
        qL[v] = tvd2(s1, s2, s3);
        qR[v] = tvd2(s4, s3, s2);
      } else {
        qL[v] = weno5(s0, s1, s2, s3, s4);
        qR[v] = weno5(s5, s4, s3, s2, s1);
      }
    }
    if (!(qL[0] > 0.0) || !(qL[3] > 0.0) || !(qR[0] > 0.0) || !(qR[3] > 0.0)) {
      for (int v = 0; v < 4; v++) {
        qL[v] = sq[v][f + 2][a];
        qR[v] = sq[v][f + 3][a];
      }
    }
    double F[4];
    // normal velocity v, tangential u
    ldfss_f64<DUAL>(qL[0], qL[2], qL[1], qL[3], qR[0], qR[2], qR[1], qR[3], k.gamma,
                    DUAL ? face_mr2(k, qL, qR, k.dy) : 1.0, F);
    const int b = f + 2, b1 = f + 3;
    const double uy = (sq[1][b1][a] - sq[1][b][a]) * idy;
    const double vy = (sq[2][b1][a] - sq[2][b][a]) * idy;
    const double Ty = (sT[b1][a] - sT[b][a]) * idy;
    const double ux = (sq[1][b][a + 1] - sq[1][b][a - 1] + sq[1][b1][a + 1] - sq[1][b1][a - 1]) * (0.25 * idx);
    const double vx = (sq[2][b][a + 1] - sq[2][b][a - 1] + sq[2][b1][a + 1] - sq[2][b1][a - 1]) * (0.25 * idx);
    const double tyy = mu * ((4.0 / 3.0) * vy - (2.0 / 3.0) * ux);
    const double txy = mu * (uy + vx);
    const double uf = 0.5 * (sq[1][b][a] + sq[1][b1][a]), vf = 0.5 * (sq[2][b][a] + sq[2][b1][a]);
    sfy[0][f][col] = F[0];
    sfy[1][f][col] = F[2] - txy;
    sfy[2][f][col] = F[1] - tyy;
    sfy[3][f][col] = F[3] - (uf * txy + vf * tyy + kap * Ty);
  }
  __syncthreads();
  if (!fluid) return;
  const long long id = cidx(k, ci, cj);
  if (!DUAL) {
    for (int v = 0; v < 4; v++) {
      const double L = -((sfx[v][ty][tx + 1] - sfx[v][ty][tx]) * idx + (sfy[v][ty + 1][tx] - sfy[v][ty][tx]) * idy);
      const long long o = id + v * P;
      double r;
      if (STAGE == 1) r = Un[o] + dt * L;
      else if (STAGE == 2) r = 0.75 * Un[o] + 0.25 * (In[o] + dt * L);
      else r = (1.0 / 3.0) * Un[o] + (2.0 / 3.0) * (In[o] + dt * L);
      Out[o] = r;
    }
    return;
  }
  // Dual time (Sec. 2): pseudo-time stage of the point-implicit preconditioned update
  //   [Gamma/dtau + a dW/dQ] dQ = -(R + BDF(W)),  a = 3/(2 dt) (BDF2) or 1/dt (first step)
  // combined with the sub-iteration's start Q0 as SSP-RK3 stage STAGE.  FP64 4x4 solve.
  const bool bdf2 = ds->steps > 0;
  const double dtp = k.dt_phys;
  double W[4], S[4];
  for (int v = 0; v < 4; v++) W[v] = In[id + v * P];
  const double r = W[0], iu = W[1] / r, iv = W[2] / r;
  const double pr = g1 * (W[3] - 0.5 * r * (iu * iu + iv * iv));
  const double T = pr / (r * k.R);
  for (int v = 0; v < 4; v++) {
    const double Rv = (sfx[v][ty][tx + 1] - sfx[v][ty][tx]) / k.dx + (sfy[v][ty + 1][tx] - sfy[v][ty][tx]) / k.dy;
    const long long o = id + v * P;
    const double tdt = bdf2 ? (3.0 * W[v] - 4.0 * Wn[o] + Wm[o]) / (2.0 * dtp) : (W[v] - Wn[o]) / dtp;
    S[v] = -(Rv + tdt);
  }
  const double cs = sqrt(k.gamma * pr / r);
  const double Vm = sqrt(iu * iu + iv * iv);
  double Ur = fmax(fmax(Vm, 1.0), k.mu / r / k.dmin);
  Ur = fmin(Ur, cs);
  const double mr2 = (Ur / cs) * (Ur / cs);
  const double up = 0.5 * Vm * (1.0 + mr2);
  const double om = 1.0 - mr2;
  const double cp_ = 0.5 * sqrt(om * om * Vm * Vm + 4.0 * Ur * Ur);
  const double vis = (2.0 * k.gamma * k.mu / k.prandtl) * (1.0 / (k.dx * k.dx) + 1.0 / (k.dy * k.dy));
  const double lam = (up + cp_) * (1.0 / k.dx + 1.0 / k.dy) + vis / r;
  const double dtau = k.cfl_tau / lam;
  const double theta = 1.0 / (Ur * Ur) - (-r / T) / (r * k.cp);
  double G[16], J[16];
  wq_matrix(theta, pr, iu, iv, T, r, k.cp, G);
  wq_matrix(1.0 / (k.R * T), pr, iu, iv, T, r, k.cp, J);
  const double a = bdf2 ? 1.5 / dtp : 1.0 / dtp;
  for (int q = 0; q < 16; q++) G[q] = G[q] / dtau + a * J[q];
  double dQ[4];
  if (!solve4(G, S, dQ)) return;
  // Q0 of the sub-iteration (held in Un = A)
  const double r0 = Un[id], u0 = Un[id + P] / r0, v0 = Un[id + 2 * P] / r0;
  const double p0 = g1 * (Un[id + 3 * P] - 0.5 * r0 * (u0 * u0 + v0 * v0));
  const double Q0[4] = {p0, u0, v0, p0 / (r0 * k.R)};
  const double Qk[4] = {pr, iu, iv, T};
  double Qn[4];
  for (int v = 0; v < 4; v++) {
    const double e = Qk[v] + dQ[v];
    Qn[v] = STAGE == 1 ? e : (STAGE == 2 ? 0.75 * Q0[v] + 0.25 * e : (1.0 / 3.0) * Q0[v] + (2.0 / 3.0) * e);
  }
  const double rn = Qn[0] / (k.R * Qn[3]);
  Out[id] = rn;
  Out[id + P] = rn * Qn[1];
  Out[id + 2 * P] = rn * Qn[2];
  Out[id + 3 * P] = Qn[0] / (k.gamma - 1.0) + 0.5 * rn * (Qn[1] * Qn[1] + Qn[2] * Qn[2]);
}

void launch_dual_f64(const Consts &k, int stage, const double *A, const double *In, double *Out, const double *Wn,
                     const double *Wm, const uint8_t *tag, DevState *ds, cudaStream_t s) {
  dim3 grid((k.nx + TX - 1) / TX, (k.ny + TY - 1) / TY);
  if (stage == 1) k_stage_f64<1, true><<<grid, 256, 0, s>>>(k, A, In, Out, Wn, Wm, tag, ds);
  else if (stage == 2) k_stage_f64<2, true><<<grid, 256, 0, s>>>(k, A, In, Out, Wn, Wm, tag, ds);
  else k_stage_f64<3, true><<<grid, 256, 0, s>>>(k, A, In, Out, Wn, Wm, tag, ds);
}

__global__ void k_dual_end(Consts k, DevState *ds) {
  ds->t = ds->t + k.dt_phys;
  ds->steps += 1;
}

void launch_dual_end(const Consts &k, DevState *ds, cudaStream_t s) { k_dual_end<<<1, 1, 0, s>>>(k, ds); }

void launch_stage_f64(const Consts &k, int stage, const double *Un, const double *In, double *Out,
                      const uint8_t *tag, DevState *ds, cudaStream_t s) {
  dim3 grid((k.nx + TX - 1) / TX, (k.ny + TY - 1) / TY);
  if (stage == 1) k_stage_f64<1, false><<<grid, 256, 0, s>>>(k, Un, In, Out, nullptr, nullptr, tag, ds);
  else if (stage == 2) k_stage_f64<2, false><<<grid, 256, 0, s>>>(k, Un, In, Out, nullptr, nullptr, tag, ds);
  else k_stage_f64<3, false><<<grid, 256, 0, s>>>(k, Un, In, Out, nullptr, nullptr, tag, ds);
}

}  // namespace ibm
