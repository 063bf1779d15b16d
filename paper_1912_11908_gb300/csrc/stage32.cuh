// Per-tile device code of the FP32-bulk stage kernels, shared by the
// single-case kernels (flow32.cu) and the block-table kernels of the
// request loop (batch32.cu), which live in separate modules.
//
// FP32-bulk flow kernels.
//
// Stage values, reconstruction and fluxes run in FP32 on perturbations from
// the free stream, dU = (rho - rho_inf, rho u - rho_inf u_inf,
// rho v - rho_inf v_inf, W'), W' = (rho E - rho_inf E_inf) - H_inf (rho -
// rho_inf).  Primitives are (rho', u, v, p') with p' = p - p_inf and
// T' = T - T_inf formed without ever adding p_inf or H_inf to an FP32 value,
// so O(M^2) pressure and temperature fluctuations keep their FP32 precision
// at any free-stream Mach number.  The state U^n is held in FP64 as the same
// perturbation dU and accumulated in FP64 at the last stage of every step:
// dU^{n+1} = dU^n + (double)[2/3 ((dU^(2) - dU^n) + dt L)], where the bracket
// is an O(dt) increment formed in FP32 (the FP32 mirror of dU^n is rounded
// from the FP64 state after every step, so FP32 rounding never accumulates in
// U^n).
#pragma once

#include <cuda.h>  // CUtensorMap

#include "dual_update.cuh"  // FP64 point-implicit update of the dual-time pseudo stages
#include "ibm_internal.cuh"

namespace ibm {

// perturbation conserved -> (rho', u, v, p', T')
__device__ __forceinline__ void pert_prim(const PertConsts &c, float dr, float dmx, float dmy, float W, float &u,
                                          float &v, float &pp, float &Tp) {
  const float r = 1.f + dr;
  const float ir = 1.f / r;
  u = (c.ux + dmx) * ir;
  v = (c.uy + dmy) * ir;
  const float du = (dmx - dr * c.ux) * ir, dv = (dmy - dr * c.uy) * ir;
  const float dq = du * (u + c.ux) + dv * (v + c.uy);  // |u|^2 - |u_inf|^2
  const float ke = 0.5f * (dr * (u * u + v * v) + dq);  // (rho |u|^2 - rho_inf |u_inf|^2) / 2
  pp = c.g1 * (W + c.Hinf * dr - ke);
  Tp = (pp - c.R * dr) * ir / c.R;
}

// (p', u, v, T') -> perturbation conserved
__device__ __forceinline__ void prim_pert(const PertConsts &c, float pp, float u, float v, float Tp, float &dr,
                                          float &dmx, float &dmy, float &W) {
  dr = (pp - c.R * Tp) / (c.R * (1.f + Tp));
  dmx = dr * u + (u - c.ux);
  dmy = dr * v + (v - c.uy);
  const float dq = (u - c.ux) * (u + c.ux) + (v - c.uy) * (v + c.uy);
  const float ke = 0.5f * (dr * (u * u + v * v) + dq);
  W = pp / c.g1 + ke - c.Hinf * dr;
}

// LDFSS(0) in perturbation form (Mr^2 = 1).  States (rho', un, ut, p');
// un_inf / ut_inf the free-stream components along the face normal and
// tangent.  Momentum flux drops the constant p_inf n (its divergence is
// zero); D_L + D_R - 1 is formed in factored form for two subsonic sides so
// p_inf (D_L + D_R - 1) keeps its precision.
//
// PRE (dual time, Sec. 2): the low-Mach numerical sound speed
// c' = 1/2 sqrt((1 - Mr^2)^2 un^2 + 4 Mr^2 c^2), Mr^2 = (Ur/c)^2 with
// Ur = min(c, max(|V|, U_ref, nu/dn)) from face averages (idn = 1/dn),
// scales the mass-flux (dissipation) part; the pressure split takes the
// physical face Mach numbers and its departure from the face mean (the
// rho c du dissipation) is scaled by c'/c, as in the FP64 path.
template <bool PRE = false>
__device__ __forceinline__ void ldfss_pert(const PertConsts &c, float drL, float unL, float utL, float ppL,
                                           float drR, float unR, float utR, float ppR, float un_inf, float ut_inf,
                                           float F[4], float idn = 0.f) {
  const float rL = 1.f + drL, rR = 1.f + drR;
  const float irL = 1.f / rL, irR = 1.f / rR;
  const float cL = sqrtf(c.gamma * (c.R + ppL) * irL), cR = sqrtf(c.gamma * (c.R + ppR) * irR);
  const float HL = c.gg * (ppL - c.R * drL) * irL +
                   0.5f * ((unL - un_inf) * (unL + un_inf) + (utL - ut_inf) * (utL + ut_inf));
  const float HR = c.gg * (ppR - c.R * drR) * irR +
                   0.5f * ((unR - un_inf) * (unR + un_inf) + (utR - ut_inf) * (utR + ut_inf));
  const float cb = 0.5f * (cL + cR);
  float cs = cb, mr2 = 1.f;
  if (PRE) {
    const float ub = 0.5f * (unL + unR), vb = 0.5f * (utL + utR);
    const float Vm = sqrtf(ub * ub + vb * vb);
    const float rb = 0.5f * (rL + rR);
    float Ur = fmaxf(fmaxf(Vm, 1.f), c.mu / rb * idn);
    Ur = fminf(Ur, cb);
    mr2 = fminf((Ur / cb) * (Ur / cb), 1.f);
    const float om = 1.f - mr2;
    cs = 0.5f * sqrtf(om * om * ub * ub + 4.f * mr2 * cb * cb);
  }
  const float ics = 1.f / cs;
  const float ML = unL * ics, MR = unR * ics;
  // the split functions' subsonic / supersonic branches as selects: alpha = 1 (0) for M >= 0 (< 0) on the
  // left, the reverse on the right; beta = -1 subsonic, 0 supersonic
  const bool subL = fabsf(ML) < 1.f, subR = fabsf(MR) < 1.f;
  const float MpL = 0.25f * (ML + 1.f) * (ML + 1.f);
  const float MmR = -0.25f * (MR - 1.f) * (MR - 1.f);
  const float CVL = subL ? MpL : fmaxf(ML, 0.f);
  const float CVR = subR ? MmR : fminf(MR, 0.f);
  const float sq = sqrtf(0.5f * (ML * ML + MR * MR)) - 1.f;
  const float Mh = subL && subR ? 0.25f * sq * sq : 0.f;
  const float dp = ppL - ppR, adp = fabsf(dp);
  const float ic2 = 0.5f * ics * ics;
  const float MhP = Mh * (1.f - (dp + adp) * ic2 * irL);
  const float MhM = Mh * (1.f - (adp - dp) * ic2 * irR);
  const float Cp = CVL - MhP, Cm = CVR + MhM;
  float DL, DR, Dm1;
  if (PRE && mr2 < 1.f) {
    // pressure split with the physical face Mach numbers
    const float icb = 1.f / cb;
    const float pML = unL * icb, pMR = unR * icb;
    const bool psL = fabsf(pML) < 1.f, psR = fabsf(pMR) < 1.f;
    const float PpL = 0.25f * (pML + 1.f) * (pML + 1.f) * (2.f - pML);
    const float PmR = 0.25f * (pMR - 1.f) * (pMR - 1.f) * (2.f + pMR);
    DL = psL ? PpL : (pML >= 0.f ? 1.f : 0.f);
    DR = psR ? PmR : (pMR >= 0.f ? 0.f : 1.f);
    Dm1 = (psL && psR) ? 0.25f * (pMR - pML) * (pMR * pMR + pMR * pML + pML * pML - 3.f) : (DL + DR - 1.f);
  } else {
    const float PpL = MpL * (2.f - ML);
    const float PmR = -MmR * (2.f + MR);
    DL = subL ? PpL : (ML >= 0.f ? 1.f : 0.f);
    DR = subR ? PmR : (MR >= 0.f ? 0.f : 1.f);
    Dm1 = (subL && subR) ? 0.25f * (MR - ML) * (MR * MR + MR * ML + ML * ML - 3.f) : (DL + DR - 1.f);
  }
  const float mL = rL * cs * Cp, mR = rR * cs * Cm;
  // p_inf (D_L + D_R - 1) + D_L p'_L + D_R p'_R; with low-Mach scaling the departure from the face mean
  // 1/2 (p'_L + p'_R) is scaled by c'/c
  F[0] = mL + mR;
  if (PRE && mr2 < 1.f)
    F[1] = mL * unL + mR * unR +
           (0.5f * (ppL + ppR) + (cs / cb) * (c.R * Dm1 + (DL - 0.5f) * ppL + (DR - 0.5f) * ppR));
  else
    F[1] = mL * unL + mR * unR + c.R * Dm1 + DL * ppL + DR * ppR;
  F[2] = mL * utL + mR * utR;
  F[3] = mL * HL + mR * HR;
}

// ---------------------------------------------------------------------------
// Fused residual + stage update in FP32 perturbation form, same tiling as
// the FP64 kernel.  Stage 3 accumulates U^{n+1} in FP64 and refreshes the
// FP32 mirror of U^{n+1}.
// ---------------------------------------------------------------------------
constexpr int TX = STAGE_TILE, TY = STAGE_TILE, HX = TX + 2 * NG, HY = TY + 2 * NG;
constexpr int NFX = 4 * TY * (TX + 1), NFY = 4 * (TY + 1) * TX;  // x-face and y-face values of a tile
constexpr int RB_MAX = 192;  // IB / ghost nodes a body tile's loaded region may hold

// Shared memory of one tile.  face holds, in turn: the TMA box of the tile's
// stage input, the stencils of the region's IB / ghost nodes (body tiles),
// the WENO face states, the face fluxes; each use ends behind a barrier
// before the next begins.
struct TileSmem {
  alignas(128) float face[2 * (NFX + NFY)];
  float sq[4][HY][HX];  // rho', u, v, p' of the loaded region
  float sT[HY][HX];     // T'
  unsigned long long mbar;
  unsigned int mbar_phase;  // persistent kernel: parity of the barrier's next phase (barrier initialised once)
  float wm[7];    // wall velocity and acceleration at the stage time; 1 if Eq. 7 applies (else 0); the rotation
                  // rate and its rate of change of a pitching body (else 0)
  float lred[8];  // per-warp maxima of the CFL reduction
  int nrb;        // listed IB / ghost nodes (body tiles)
  int rbm[RB_MAX], rbe[RB_MAX];
};
static_assert(RB_MAX * sizeof(RStencil32) <= sizeof(float) * 2 * (NFX + NFY), "node stencils fit the face storage");

// ---------------------------------------------------------------------------
// TMA staging of a tile (Blackwell bulk tensor copy, inline PTX).  The FP32
// arrays are 3-D tensors (padded column, padded row, variable plane); the
// loaded region of an interior tile is the box of TMA_W x HY x 4 floats at
// padded (i0, j0, 0) -- i0 is a multiple of the tile width, so the copy
// starts on a 64-byte boundary.  One elected thread arms an mbarrier with the
// box's byte count and issues the copy; the block waits on the barrier.
// ---------------------------------------------------------------------------
constexpr int TMA_W = (HX + 3) / 4 * 4;  // box width: HX rounded up to a multiple of 16 bytes
constexpr unsigned TMA_BYTES = 4u * HY * TMA_W * sizeof(float);
// a tile's copy completes within microseconds; a wait gives up after about a second of %globaltimer (the
// iteration count is only a backstop: the time a try_wait suspends is implementation-defined)
constexpr unsigned long long TMA_WAIT_NS = 1ull << 30;
constexpr unsigned TMA_WAIT_BACKSTOP = 1u << 28;

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tma_init(unsigned long long *mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// arm the (initialised) barrier with the box's byte count and issue the copy
__device__ __forceinline__ void tma_load(float *dst, const CUtensorMap *map, int x, int y, unsigned long long *mbar) {
  const unsigned m = smem_u32(mbar);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(m), "r"(TMA_BYTES) : "memory");
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(smem_u32(dst)),
      "l"((unsigned long long)map), "r"(x), "r"(y), "r"(0), "r"(m)
      : "memory");
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// wait for the completion of the barrier's phase with the given parity; false if it has not completed within
// TMA_WAIT_NS
__device__ __forceinline__ bool tma_wait(unsigned long long *mbar, unsigned parity) {
  const unsigned m = smem_u32(mbar);
  unsigned long long t0 = 0;
  for (unsigned it = 0; it < TMA_WAIT_BACKSTOP; it++) {
    unsigned ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(m), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 63) == 0) {
      const unsigned long long t = globaltimer_ns();
      if (it == 0) t0 = t;
      else if (t - t0 > TMA_WAIT_NS) return false;
    }
  }
  return false;
}

// spectral radius of the CFL rule for one cell of the FP32 mirror
__device__ __forceinline__ float cfl_lambda(const Consts &k, const PertConsts &c, const float m[4]) {
  float u, v, pp, Tp;
  pert_prim(c, m[0], m[1], m[2], m[3], u, v, pp, Tp);
  const float r = 1.f + m[0];
  const float cs = sqrtf(c.gamma * (c.R + pp) / r);
  return (fabsf(u) + cs) * c.idx + (fabsf(v) + cs) * c.idy + c.vis / r;
}

// block maximum of lam (all 256 threads call), then the grid-wide maximum and
// dt through the last-block pattern
__device__ __forceinline__ void cfl_block_max(const Consts &k, float lam, float *red, DevState *ds,
                                              unsigned int nblocks, bool defer) {
  for (int off = 16; off > 0; off >>= 1) lam = fmaxf(lam, __shfl_xor_sync(0xffffffffu, lam, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = lam;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = red[0];
    for (int w = 1; w < 8; w++) m = fmaxf(m, red[w]);
    atomicMax(&ds->lmax_bits, (unsigned long long)__double_as_longlong((double)m));
    finish_cfl(k, ds, nblocks, defer);
  }
}

// load of a value that other blocks of the same launch may have written (CG:
// through L2, never the non-coherent read-only path)
template <bool CG, class T>
__device__ __forceinline__ T ld_stage(const T *p) {
  if (CG) return __ldcg(p);
  return *p;
}

// ---------------------------------------------------------------------------
// IB / ghost reconstruction (Sec. 4.4-4.6, Eq. 4-8; Sec. 5) evaluated while a
// tile is loaded.  Values are primitives (p', u, v, T').  A ghost node's
// image point may use IB nodes, which are rebuilt from their own stencils
// (their corners are fluid): a body tile rebuilds all IB nodes of its loaded
// region, then all ghost nodes, reading corners from shared memory and only
// corners outside the region from the stage input.
// ---------------------------------------------------------------------------
template <bool CG = false>
__device__ __forceinline__ void raw_prim(const PertConsts &c, const float *U, long long id, long long P,
                                         float q[4]) {
  float u, v, pp, Tp;
  pert_prim(c, ld_stage<CG>(U + id), ld_stage<CG>(U + id + P), ld_stage<CG>(U + id + 2 * P),
            ld_stage<CG>(U + id + 3 * P), u, v, pp, Tp);
  q[0] = pp;
  q[1] = u;
  q[2] = v;
  q[3] = Tp;
}

__device__ __forceinline__ void wall_bc(const PertConsts &c, const RStencil32 &s, const float qp[4], const float *wm,
                                        float q[4]) {
  // wm = (Vx, Vy, Ax, Ay, supersonic, omega, domega/dt) at the stage time: the wall's motion at P' is the
  // body's translation plus, for a pitching body, omega x r and domega/dt x r - omega^2 r with r = P' - pivot
  // (zero terms otherwise).  Neumann pressure dp/dn = rho G (Eq. 5-6), G = -n.a plus the centripetal
  // u_t^2 kappa of Eq. 7 (u_t tangential to the wall, relative to it, at the probe); with rho = p / (R T) and
  // T fixed along the normal (Eq. 8) it integrates to p = p_probe exp(-dxi G / (R T)), here in perturbation
  // form p' = p'_probe + (R + p'_probe) expm1(...) so that p' keeps its digits
  const float om = wm[5], al = wm[6];
  const float Vx = wm[0] - om * s.ry, Vy = wm[1] + om * s.rx;
  const float Ax = wm[2] - al * s.ry - om * om * s.rx, Ay = wm[3] + al * s.rx - om * om * s.ry;
  float G = -(s.nx * Ax + s.ny * Ay);
  if (wm[4] != 0.f) {
    const float ut = -(qp[1] - Vx) * s.ny + (qp[2] - Vy) * s.nx;
    G = G + ut * ut * s.curv;
  }
  // (static body: G = 0 and p'_node = p'_probe exactly, without the exponential)
  q[0] = G != 0.f ? qp[0] + (c.R + qp[0]) * expm1f(-s.dxi * G / (c.R * (1.f + qp[3]))) : qp[0];
  q[1] = Vx + (qp[1] - Vx) * s.ratio;
  q[2] = Vy + (qp[2] - Vy) * s.ratio;
  q[3] = qp[3];
}

// The quadratic form (Sec. 4.5, Sec. 5; IBM_INTERP_QUADRATIC) of wall_bc: quadratics in the distance along the
// normal through the wall condition and the probes' values qp (first) and qb (second) -- the Lagrange weights
// for the Dirichlet velocity, zero wall slope for T', wall slope rho G for p' with the first probe's density --
// in perturbation form (differences of perturbations are differences of the variables)
__device__ __forceinline__ void wall_bc_quad(const PertConsts &c, const RStencil32 &s, const RStencilQ &t,
                                             const float qp[4], const float qb[4], const float *wm, float q[4]) {
  const float om = wm[5], al = wm[6];
  const float Vx = wm[0] - om * s.ry, Vy = wm[1] + om * s.rx;
  const float Ax = wm[2] - al * s.ry - om * om * s.rx, Ay = wm[3] + al * s.rx - om * om * s.ry;
  float G = -(s.nx * Ax + s.ny * Ay);
  if (wm[4] != 0.f) {
    const float ut = -(qp[1] - Vx) * s.ny + (qp[2] - Vy) * s.nx;
    G = G + ut * ut * s.curv;
  }
  const float b = (c.R + qp[0]) / (c.R * (1.f + qp[3])) * G;
  q[0] = qp[0] + (qb[0] - qp[0]) * t.m + b * t.dq;
  q[1] = Vx + (qp[1] - Vx) * t.L1 + (qb[1] - Vx) * t.L2;
  q[2] = Vy + (qp[2] - Vy) * t.L1 + (qb[2] - Vy) * t.L2;
  q[3] = qp[3] + (qb[3] - qp[3]) * t.m;
}

// An IB node outside a tile's loaded region, rebuilt from its own stencil (QUAD: and its second probe)
template <bool CG, bool QUAD = false>
static __device__ __noinline__ void rebuild_ib(const Consts &k, const PertConsts &c, const float *U,
                                               const RStencil32 &s, const RStencilQ *t, const float *wm,
                                               float q[4]) {
  float qp[4] = {0.f, 0.f, 0.f, 0.f};
  for (int b = 0; b < 4; b++) {
    if (!(s.mask >> b & 1)) continue;  // bits 0-3: valid corners (bit 4: IB node)
    float cq[4];
    raw_prim<CG>(c, U, s.corner + (b & 1) + (b >> 1) * k.pitch, k.plane, cq);
    for (int v = 0; v < 4; v++) qp[v] += s.w[b] * cq[v];
  }
  if (QUAD && t->mask) {
    float qb[4] = {0.f, 0.f, 0.f, 0.f};
    for (int b = 0; b < 4; b++) {
      if (!(t->mask >> b & 1)) continue;
      float cq[4];
      raw_prim<CG>(c, U, t->corner + (b & 1) + (b >> 1) * k.pitch, k.plane, cq);
      for (int v = 0; v < 4; v++) qb[v] += t->w[b] * cq[v];
    }
    wall_bc_quad(c, s, *t, qp, qb, wm, q);
  } else {
    wall_bc(c, s, qp, wm, q);
  }
}

// ---------------------------------------------------------------------------
// Fused residual + stage update in FP32 perturbation form.  One 16x16 tile
// per block.  (1) Load tile + 3-cell halo: domain halos by index mapping, IB
// and ghost nodes rebuilt on the fly, conversion to (rho', u, v, p', T') in
// shared memory.  (2) WENO5 per cell and direction: the three smoothness
// indicators of a cell's five-point window serve both the left state of its
// right face and the right state of its left face.  (3) LDFSS + central
// viscous flux per face.  (4) Flux divergence and SSP-RK3 stage update;
// stage 3 accumulates U^{n+1} in FP64.
// ---------------------------------------------------------------------------
// blk: the block's index within this case's launch (plain: tile index; body:
// slot in the body-tile list).  Every thread of the block calls it.
// DUAL: a pseudo stage of dual time -- preconditioned faces, wall motion at
// t + dt_phys, FP64 point-implicit update (dp; D holds the sub-iteration's
// start, Out receives the FP32 mirror of the new iterate).
// TMA: the kernel may stage interior tiles with a tensor copy (tmap: tensor
// map of In; NULL loads every tile with per-thread loads).
// PERSIST: the tile's stage inside the persistent step kernel -- blk is the
// tile itself; In, D and the stage arrays may have been written by other
// blocks of the same launch (coherent loads); stage times come from t and dt,
// which stay fixed during the launch; the step's end (t, step count) and the
// next dt are left to the kernel.
// sm: the block's shared memory.
// TVD: the second-order TVD reconstruction in place of WENO5 (Sec. 2), compiled into its own kernels so that
// the WENO5 kernels carry no branch for it.
template <int STAGE, bool BODY, bool DUAL = false, bool TMA = false, bool PERSIST = false, bool TVD = false,
          bool QUAD = false>
__device__ __forceinline__ void stage_tile(const Consts &k, const PertConsts &c, float *Mn,
                                           const float *__restrict__ In, float *Out, double *D,
                                           const uint8_t *__restrict__ tag,
                                           const int *__restrict__ sid, const RStencil32 *__restrict__ rs,
                                           const uint8_t *__restrict__ tile_body, const int *__restrict__ body_tiles,
                                           DevState *ds, bool fuse_cfl, unsigned int ncfl, int blk, TileSmem &sm,
                                           const DualPtrs &dp = DualPtrs{}, const CUtensorMap *tmap = nullptr,
                                           const RStencilQ *__restrict__ rsq = nullptr) {
  static_assert(!TMA || 4 * HY * TMA_W <= 2 * (NFX + NFY), "TMA box must fit in the face-state storage");
  float *s_face = sm.face;
  unsigned long long &s_mbar = sm.mbar;
  float(&sq)[4][HY][HX] = sm.sq;
  float(&sT)[HY][HX] = sm.sT;
  float(*fLx)[TY][TX + 1] = reinterpret_cast<float(*)[TY][TX + 1]>(s_face);  // x-face states; fLx then x flux
  float(*fRx)[TY][TX + 1] = reinterpret_cast<float(*)[TY][TX + 1]>(s_face + NFX);
  float(*fLy)[TY + 1][TX] = reinterpret_cast<float(*)[TY + 1][TX]>(s_face + 2 * NFX);  // y-face states; then y flux
  float(*fRy)[TY + 1][TX] = reinterpret_cast<float(*)[TY + 1][TX]>(s_face + 2 * NFX + NFY);
  float(*s_raw)[HY][TMA_W] = reinterpret_cast<float(*)[HY][TMA_W]>(s_face);  // TMA box
  float *wm = sm.wm;
  float *lred = sm.lred;
  const int ntx = (k.nx + TX - 1) / TX;
  // every block reads dt before any block can finish the fused CFL reduction
  const double dtd = ds->dt;
  const float dt = ds->dtf;
  int tile;
  if (PERSIST) {
    tile = blk;
  } else if (BODY) {
    tile = blk < ds->nbody_tiles ? body_tiles[blk] : -1;
  } else {
    tile = tile_body[blk] ? -1 : blk;
    if (!DUAL && blk == 0 && threadIdx.x == 0) {
      if (STAGE == 1) {  // stage times for the body kernels of stages 2 and 3
        ds->tst[0] = ds->t + dtd;
        ds->tst[1] = ds->t + 0.5 * dtd;
      } else if (STAGE == 3) {  // end of the step; the body kernel of stage 3 reads tst, not t
        ds->t = ds->t + dtd;
        ds->steps += 1;
      }
    }
  }
  if (tile < 0) {
    if (STAGE == 3 && fuse_cfl && threadIdx.x == 0) finish_cfl(k, ds, ncfl, PERSIST);
    return;
  }
  const int i0 = (tile % ntx) * TX, j0 = (tile / ntx) * TY;
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int ci = i0 + tx, cj = j0 + ty;
  const bool inside = ci < k.nx && cj < k.ny;
  const uint8_t mytag = inside ? tag[cj * k.nx + ci] : (uint8_t)SOLID;
  // cells the flux update advances: fluid cells, and IB nodes when the ghost layers alone impose the wall
  const bool fluid = mytag == FLUID || (k.ib_advance && mytag == IB);
  // stages 1 and 3 also keep the IB / ghost nodes of U^n current; stage 2 only needs fluid cells
  const bool work = STAGE == 2 ? fluid : (mytag != SOLID);
  if (!__syncthreads_or(work)) {
    if (STAGE == 3 && fuse_cfl && threadIdx.x == 0) finish_cfl(k, ds, ncfl, PERSIST);
    return;
  }
  // L2 prefetch of the operands the stage update reads at the end of the tile (the mirror of U^n; the stage
  // input; the FP64 master at stage 3): one line per tile row and plane, issued before the tile's arithmetic
  // so that those reads find L2 rather than DRAM after the L2 has turned over
  if (!DUAL && threadIdx.x < 4 * TY) {
    const int r = threadIdx.x % TY, v = threadIdx.x / TY;
    if (j0 + r < k.ny) {
      const long long o = cidx(k, i0, j0 + r) + v * k.plane;
      asm volatile("prefetch.global.L2 [%0];" ::"l"(Mn + o));
      if (STAGE >= 2) asm volatile("prefetch.global.L2 [%0];" ::"l"(In + o));
      if (STAGE == 3) {
        asm volatile("prefetch.global.L2 [%0];" ::"l"(D + o));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(D + o + 8));
      }
    }
  }
  if (BODY && threadIdx.x == 0) {
    double X[2], V[2], Acc[2];
    const double ts = DUAL ? ds->t + k.dt_phys
                           : (PERSIST ? stage_time(ds, STAGE) : (STAGE == 1 ? ds->t : ds->tst[STAGE - 2]));
    body_motion(k, ds, ts, X, V, Acc);
    wm[0] = (float)V[0];
    wm[1] = (float)V[1];
    wm[2] = (float)Acc[0];
    wm[3] = (float)Acc[1];
    wm[4] = supersonic_motion(k, V) ? 1.f : 0.f;
    double th = 0.0, om = 0.0, al = 0.0;
    if (k.motion.kind == IBM_MOTION_PITCH) pitch_at(k.motion, ts, &th, &om, &al);
    wm[5] = (float)om;
    wm[6] = (float)al;
  }
  // interior tile (the loaded region needs no domain mapping): one tensor copy stages it
  const bool tma = TMA && tmap != nullptr && i0 >= NG && j0 >= NG && i0 + TX + NG <= k.nx && j0 + TY + NG <= k.ny;
  if (TMA && tma && threadIdx.x == 0) {
    if (PERSIST) {
      // the box may hold values other blocks of this launch wrote: order the tensor copy after them
      asm volatile("fence.proxy.async.global;" ::: "memory");
    } else {
      tma_init(&s_mbar);
    }
    tma_load(s_face, tmap, i0, j0, &s_mbar);
  }
  __syncthreads();
  if (TMA && tma) {
    const unsigned parity = PERSIST ? sm.mbar_phase : 0u;
    if (__syncthreads_or(!tma_wait(&s_mbar, parity))) {
      // the copy has not completed and may still write the box: wait for it once more (bounded), then leave
      // the tile without touching shared memory or outputs.  The step's state is invalid; the error flag makes
      // the next synchronising call report it.
      if (threadIdx.x == 0) {
        atomicOr(&ds->err, ERR_TIMEOUT);
        tma_wait(&s_mbar, parity);
        if (STAGE == 3 && fuse_cfl) finish_cfl(k, ds, ncfl, PERSIST);
      }
      return;
    }
  }

  const long long P = k.plane;
  // body tiles: every IB / ghost node of the loaded region, with its stencil staged in shared memory (in the
  // face storage, after the TMA box has been consumed)
  int &s_nrb = sm.nrb;
  int *s_rbm = sm.rbm, *s_rbe = sm.rbe;
  RStencil32 *s_rs = reinterpret_cast<RStencil32 *>(s_face);
  if (BODY && threadIdx.x == 0) s_nrb = 0;
  if (BODY) __syncthreads();
  for (int m = threadIdx.x; m < HX * HY; m += 256) {
    const int a = m % HX, b = m / HX;
    int gi = i0 - NG + a, gj = j0 - NG + b;
    float q[4] = {0.f, c.ux, c.uy, 0.f};  // (p', u, v, T'); free stream: zero perturbation
    float dr = 0.f;
    if (TMA && tma) {
      float u, v, pp, Tp;
      dr = s_raw[0][b][a];
      pert_prim(c, dr, s_raw[1][b][a], s_raw[2][b][a], s_raw[3][b][a], u, v, pp, Tp);
      q[0] = pp;
      q[1] = u;
      q[2] = v;
      q[3] = Tp;
      if (BODY) {
        const int e = sid[gj * k.nx + gi];
        if (e >= 0) {
          const int slot = atomicAdd(&s_nrb, 1);
          if (slot < RB_MAX) {
            s_rbm[slot] = m;
            s_rbe[slot] = e;
          }
        }
      }
    } else if (halo_map(k, gi, gj)) {
      const long long id = cidx(k, gi, gj);
      int e = -1;
      if (BODY) e = sid[gj * k.nx + gi];
      dr = ld_stage<PERSIST>(In + id);
      raw_prim<PERSIST>(c, In, id, P, q);
      if (BODY && e >= 0) {
        const int slot = atomicAdd(&s_nrb, 1);
        if (slot < RB_MAX) {
          s_rbm[slot] = m;
          s_rbe[slot] = e;
        }
      }
    }
    sq[0][b][a] = dr;
    sq[1][b][a] = q[1];
    sq[2][b][a] = q[2];
    sq[3][b][a] = q[0];
    sT[b][a] = q[3];
  }
  __syncthreads();
  // every thread has waited on this phase: the next tile's copy completes the other parity
  if (PERSIST && TMA && tma && threadIdx.x == 0) sm.mbar_phase ^= 1u;
  if (BODY) {
    const int nrb = min(s_nrb, RB_MAX);
    for (int r = threadIdx.x; r < nrb; r += 256) s_rs[r] = rs[s_rbe[r]];
    __syncthreads();
    // rebuild the listed nodes in place: IB nodes, barrier, ghost nodes (whose image points may use IB
    // nodes); corners inside the loaded region come from shared memory
    // four lanes per node, one stencil corner each, so that corners outside the loaded region (chains of
    // dependent global loads) overlap; the node's first lane sums the corners in stencil order
    for (int pass = k.ib_advance ? 1 : 0; pass < 2; pass++) {  // IB nodes (pass 0) unless advanced
      for (int t0 = 0; t0 < 4 * nrb; t0 += 256) {  // block-uniform: every lane takes part in the shuffles
        const int r = (t0 + (int)threadIdx.x) >> 2, cq = threadIdx.x & 3;
        bool node = false;
        float v4[4] = {0.f, 0.f, 0.f, 0.f};
        if (r < nrb) {
          const RStencil32 &st = s_rs[r];
          node = ((st.mask & 16) != 0) == (pass == 0) && (st.mask & 15);
          if (node && (st.mask >> cq & 1)) {
            const int cn = st.ccell + (cq & 1) + (cq >> 1) * k.nx;
            const int la = cn % k.nx - (i0 - NG), lb = cn / k.nx - (j0 - NG);
            if (la >= 0 && la < HX && lb >= 0 && lb < HY) {
              v4[0] = sq[3][lb][la];
              v4[1] = sq[1][lb][la];
              v4[2] = sq[2][lb][la];
              v4[3] = sT[lb][la];
            } else {
              // corner outside the loaded region: fluid value, or an IB node rebuilt from its own stencil
              const int e2 = pass == 1 ? sid[cn] : -1;
              if (!k.ib_advance && e2 >= 0 && (rs[e2].mask & 15))
                rebuild_ib<PERSIST, QUAD>(k, c, In, rs[e2], QUAD ? rsq + e2 : nullptr, wm, v4);
              else raw_prim<PERSIST>(c, In, st.corner + (cq & 1) + (cq >> 1) * k.pitch, P, v4);
            }
          }
        }
        // quadratic form: the same lane also takes its corner of the second probe's square
        const RStencilQ *tq = nullptr;
        float v4b[4] = {0.f, 0.f, 0.f, 0.f};
        if (QUAD && r < nrb && node) {
          tq = rsq + s_rbe[r];
          if (tq->mask >> cq & 1) {
            const int cn = tq->ccell + (cq & 1) + (cq >> 1) * k.nx;
            const int la = cn % k.nx - (i0 - NG), lb = cn / k.nx - (j0 - NG);
            if (la >= 0 && la < HX && lb >= 0 && lb < HY) {
              v4b[0] = sq[3][lb][la];
              v4b[1] = sq[1][lb][la];
              v4b[2] = sq[2][lb][la];
              v4b[3] = sT[lb][la];
            } else {
              const int e2 = pass == 1 ? sid[cn] : -1;
              if (!k.ib_advance && e2 >= 0 && (rs[e2].mask & 15))
                rebuild_ib<PERSIST, QUAD>(k, c, In, rs[e2], rsq + e2, wm, v4b);
              else raw_prim<PERSIST>(c, In, tq->corner + (cq & 1) + (cq >> 1) * k.pitch, P, v4b);
            }
          }
        }
        const int lane0 = (int)(threadIdx.x & 31) & ~3;
        float qp[4] = {0.f, 0.f, 0.f, 0.f};
        const unsigned int mask = r < nrb ? (unsigned int)s_rs[r].mask : 0u;
        for (int j = 0; j < 4; j++) {
          const float wj = r < nrb ? s_rs[r].w[j] : 0.f;
          for (int v = 0; v < 4; v++) {
            const float x = __shfl_sync(0xffffffffu, v4[v], lane0 + j);
            if (mask >> j & 1) qp[v] += wj * x;
          }
        }
        float qb[4] = {0.f, 0.f, 0.f, 0.f};
        if (QUAD) {
          const unsigned int maskb = tq ? (unsigned int)tq->mask : 0u;
          for (int j = 0; j < 4; j++) {
            const float wj = tq ? tq->w[j] : 0.f;
            for (int v = 0; v < 4; v++) {
              const float x = __shfl_sync(0xffffffffu, v4b[v], lane0 + j);
              if (maskb >> j & 1) qb[v] += wj * x;
            }
          }
        }
        if (!node || cq != 0) continue;
        const RStencil32 &st = s_rs[r];
        const int m = s_rbm[r], a = m % HX, b = m / HX;
        float q[4];
        if (QUAD && tq->mask) wall_bc_quad(c, st, *tq, qp, qb, wm, q);
        else wall_bc(c, st, qp, wm, q);
        sq[0][b][a] = (q[0] - c.R * q[3]) / (c.R * (1.f + q[3]));
        sq[1][b][a] = q[1];
        sq[2][b][a] = q[2];
        sq[3][b][a] = q[0];
        sT[b][a] = q[3];
        const bool own = a >= NG && a < NG + TX && b >= NG && b < NG + TY;
        if (own && STAGE == 1) {  // U^n on this node for output and for a node that turns fluid
          float d0, d1, d2, d3;
          prim_pert(c, q[0], q[1], q[2], q[3], d0, d1, d2, d3);
          D[st.cell] = d0;
          D[st.cell + P] = d1;
          D[st.cell + 2 * P] = d2;
          D[st.cell + 3 * P] = d3;
        }
      }
      __syncthreads();
    }
    if (threadIdx.x == 0 && s_nrb > RB_MAX) atomicOr(&ds->err, ERR_CAPACITY);
  }
  // WENO5 (Sec. 2) along lines: an item is one variable of one interior tile row (x) or column (y) and one of
  // its two halves -- nine consecutive window centres, local 2..10 or 11..19, the cells whose faces the tile
  // needs.  The smoothness indicators are written with the second differences d2 and first differences g of the
  // line, beta_0 = 13/12 d2(c-1)^2 + 1/4 (d2(c-1) + 2 g(c-1))^2, beta_1 = 13/12 d2(c)^2 + 1/4 (g(c-1) + g(c))^2,
  // beta_2 = 13/12 d2(c+1)^2 + 1/4 (d2(c+1) - 2 g(c))^2 with g(j) = f(j+1) - f(j), so that each centre loads one
  // value and forms one new squared second difference, shared by three windows.  The three candidate
  // polynomials and the nonlinear weights of a window give the left state at its right face and, mirrored, the
  // right state at its left face.
  static_assert(TX == 16 && TY == 16, "one item per thread: 2 directions x 16 lines x 4 variables x 2 halves");
  if (TVD) {
    // the second-order TVD scheme (Sec. 2): MUSCL with the minmod limiter over the same items; differences
    // of perturbations equal differences of the variables, so the limiter sees what it would in absolute form
    const int u = threadIdx.x & 127;
    const bool xdir = threadIdx.x < 128;
    const int half = u & 1, line = (u >> 1) & 15, v = u >> 5;
    const float *lp = xdir ? &sq[v][NG + line][0] : &sq[v][0][NG + line];
    const int ls = xdir ? 1 : HX;
    const int p0 = 2 + 9 * half;
    float f1 = lp[(p0 - 1) * ls], f2 = lp[p0 * ls];
#pragma unroll
    for (int i = 0; i < 9; i++) {
      const int pc = p0 + i;
      const float f3 = lp[(pc + 1) * ls];
      const float a = f2 - f1, b = f3 - f2;
      // minmod(a, b) for the left state at the right face, minmod(-b, -a) = -minmod(a, b) for the right state
      float m = 0.f;
      if (a > 0.f && b > 0.f) m = a < b ? a : b;
      else if (a < 0.f && b < 0.f) m = a > b ? a : b;
      const float qL = f2 + 0.5f * m, qR = f2 - 0.5f * m;
      if (xdir) {
        if (pc - 2 <= TX) fLx[v][line][pc - 2] = qL;
        if (pc >= 3) fRx[v][line][pc - 3] = qR;
      } else {
        if (pc - 2 <= TY) fLy[v][pc - 2][line] = qL;
        if (pc >= 3) fRy[v][pc - 3][line] = qR;
      }
      f1 = f2;
      f2 = f3;
    }
  } else {
    const int u = threadIdx.x & 127;
    const bool xdir = threadIdx.x < 128;
    const int half = u & 1, line = (u >> 1) & 15, v = u >> 5;
    const float *lp = xdir ? &sq[v][NG + line][0] : &sq[v][0][NG + line];
    const int ls = xdir ? 1 : HX;  // stride along the line
    const int p0 = 2 + 9 * half;
    // the indicators are written as e_k = eps + beta_k = [eps + 13/12 d2^2] + (b_k / 2)^2: eps rides in the
    // sliding 13/12 d2^2 terms and the first-difference combinations are halved, so each e_k is one FMA
    const float eps = 1e-6f;
    float f0 = lp[(p0 - 2) * ls], f1 = lp[(p0 - 1) * ls], f2 = lp[p0 * ls], f3 = lp[(p0 + 1) * ls];
    float d2m = f0 - 2.f * f1 + f2, d2c = f1 - 2.f * f2 + f3;  // second differences centred at c - 1 and c
    float am = fmaf((13.f / 12.f) * d2m, d2m, eps), ac = fmaf((13.f / 12.f) * d2c, d2c, eps);
#pragma unroll
    for (int i = 0; i < 9; i++) {
      const int pc = p0 + i;
      const float f4 = lp[(pc + 2) * ls];
      const float d2p = f2 - 2.f * f3 + f4, ap = fmaf((13.f / 12.f) * d2p, d2p, eps);
      const float gm = f2 - f1, g0 = f3 - f2;
      const float hb0 = fmaf(0.5f, d2m, gm), hb1 = 0.5f * (gm + g0), hb2 = fmaf(0.5f, d2p, -g0);
      const float e0 = fmaf(hb0, hb0, am), e1 = fmaf(hb1, hb1, ac), e2 = fmaf(hb2, hb2, ap);
      const float e01 = e0 * e1, e12 = e1 * e2, e02 = e0 * e2;
      const float s01 = e01 * e01, s12 = e12 * e12, s02 = e02 * e02;
      // left state at the cell's right face: the candidates (2 f0 - 7 f1 + 11 f2, -f1 + 5 f2 + 2 f3,
      // 2 f2 + 5 f3 - f4) / 6 with the linear weights (0.1, 0.6, 0.3) folded into their coefficients, the
      // nonlinear weights d_k / e_k^2 cleared of their common denominator (s12 for k = 0, s02, s01)
      const float hf2 = 0.5f * f2;
      const float l0 = (1.f / 30.f) * f0 - (7.f / 60.f) * f1 + (11.f / 60.f) * f2;
      const float l1 = fmaf(-0.1f, f1, fmaf(0.2f, f3, hf2));
      const float l2 = 0.1f * f2 + 0.25f * f3 - 0.05f * f4;
      const float qL = __fdividef(fmaf(s12, l0, fmaf(s02, l1, s01 * l2)),
                                  fmaf(0.1f, s12, fmaf(0.6f, s02, 0.3f * s01)));
      // right state at the cell's left face: mirrored window, indicators reversed
      const float r0 = (1.f / 30.f) * f4 - (7.f / 60.f) * f3 + (11.f / 60.f) * f2;
      const float r1 = fmaf(-0.1f, f3, fmaf(0.2f, f1, hf2));
      const float r2 = 0.1f * f2 + 0.25f * f1 - 0.05f * f0;
      const float qR = __fdividef(fmaf(s01, r0, fmaf(s02, r1, s12 * r2)),
                                  fmaf(0.1f, s01, fmaf(0.6f, s02, 0.3f * s12)));
      if (xdir) {
        if (pc - 2 <= TX) fLx[v][line][pc - 2] = qL;  // face between pc and pc+1
        if (pc >= 3) fRx[v][line][pc - 3] = qR;        // face between pc-1 and pc
      } else {
        if (pc - 2 <= TY) fLy[v][pc - 2][line] = qL;
        if (pc >= 3) fRy[v][pc - 3][line] = qR;
      }
      f0 = f1;
      f1 = f2;
      f2 = f3;
      f3 = f4;
      d2m = d2c;
      d2c = d2p;
      am = ac;
      ac = ap;
    }
  }
  __syncthreads();

  const float mu = c.mu, kap = c.kappa, idx = c.idx, idy = c.idy;
  for (int m = threadIdx.x; m < (TX + 1) * TY + TX * (TY + 1); m += 256) {
    const bool xdir = m < (TX + 1) * TY;
    float qL[4], qR[4], F[4];
    if (xdir) {
      const int f = m % (TX + 1), row = m / (TX + 1);
      const int b = row + NG, a = f + 2, a1 = f + 3;
      for (int v = 0; v < 4; v++) {
        qL[v] = fLx[v][row][f];
        qR[v] = fRx[v][row][f];
      }
      if (!(qL[0] > -1.f) || !(qL[3] > -c.R) || !(qR[0] > -1.f) || !(qR[3] > -c.R)) {
        for (int v = 0; v < 4; v++) {
          qL[v] = sq[v][b][a];
          qR[v] = sq[v][b][a1];
        }
      }
      ldfss_pert<DUAL>(c, qL[0], qL[1], qL[2], qL[3], qR[0], qR[1], qR[2], qR[3], c.ux, c.uy, F, idx);
      const float ux = (sq[1][b][a1] - sq[1][b][a]) * idx;
      const float vx = (sq[2][b][a1] - sq[2][b][a]) * idx;
      const float Tx = (sT[b][a1] - sT[b][a]) * idx;
      const float uy = (sq[1][b + 1][a] - sq[1][b - 1][a] + sq[1][b + 1][a1] - sq[1][b - 1][a1]) * (0.25f * idy);
      const float vy = (sq[2][b + 1][a] - sq[2][b - 1][a] + sq[2][b + 1][a1] - sq[2][b - 1][a1]) * (0.25f * idy);
      const float txx = mu * ((4.f / 3.f) * ux - (2.f / 3.f) * vy);
      const float txy = mu * (uy + vx);
      const float uf = 0.5f * (sq[1][b][a] + sq[1][b][a1]), vf = 0.5f * (sq[2][b][a] + sq[2][b][a1]);
      fLx[0][row][f] = F[0];
      fLx[1][row][f] = F[1] - txx;
      fLx[2][row][f] = F[2] - txy;
      fLx[3][row][f] = F[3] - (uf * txx + vf * txy + kap * Tx);
    } else {
      const int mm = m - (TX + 1) * TY;
      const int col = mm % TX, f = mm / TX;
      const int a = col + NG, b = f + 2, b1 = f + 3;
      for (int v = 0; v < 4; v++) {
        qL[v] = fLy[v][f][col];
        qR[v] = fRy[v][f][col];
      }
      if (!(qL[0] > -1.f) || !(qL[3] > -c.R) || !(qR[0] > -1.f) || !(qR[3] > -c.R)) {
        for (int v = 0; v < 4; v++) {
          qL[v] = sq[v][b][a];
          qR[v] = sq[v][b1][a];
        }
      }
      ldfss_pert<DUAL>(c, qL[0], qL[2], qL[1], qL[3], qR[0], qR[2], qR[1], qR[3], c.uy, c.ux, F, idy);
      const float uy = (sq[1][b1][a] - sq[1][b][a]) * idy;
      const float vy = (sq[2][b1][a] - sq[2][b][a]) * idy;
      const float Ty = (sT[b1][a] - sT[b][a]) * idy;
      const float ux = (sq[1][b][a + 1] - sq[1][b][a - 1] + sq[1][b1][a + 1] - sq[1][b1][a - 1]) * (0.25f * idx);
      const float vx = (sq[2][b][a + 1] - sq[2][b][a - 1] + sq[2][b1][a + 1] - sq[2][b1][a - 1]) * (0.25f * idx);
      const float tyy = mu * ((4.f / 3.f) * vy - (2.f / 3.f) * ux);
      const float txy = mu * (uy + vx);
      const float uf = 0.5f * (sq[1][b][a] + sq[1][b1][a]), vf = 0.5f * (sq[2][b][a] + sq[2][b1][a]);
      fLy[0][f][col] = F[0];
      fLy[1][f][col] = F[2] - txy;
      fLy[2][f][col] = F[1] - tyy;
      fLy[3][f][col] = F[3] - (uf * txy + vf * tyy + kap * Ty);
    }
  }
  __syncthreads();

  float lam = 0.f;
  const long long id = cidx(k, ci, cj);
  if (fluid) {
    float L[4];
    for (int v = 0; v < 4; v++)
      L[v] = -((fLx[v][ty][tx + 1] - fLx[v][ty][tx]) * idx + (fLy[v][ty + 1][tx] - fLy[v][ty][tx]) * idy);
    if (DUAL) {
      dual_update_cell<STAGE>(k, c, id, P, L, dp, Out, ds->steps > 0);
    } else if (STAGE == 1) {
      for (int v = 0; v < 4; v++) Out[id + v * P] = Mn[id + v * P] + dt * L[v];
    } else if (STAGE == 2) {
      for (int v = 0; v < 4; v++)
        Out[id + v * P] = 0.75f * Mn[id + v * P] + 0.25f * (ld_stage<PERSIST>(In + id + v * P) + dt * L[v]);
    } else {
      // FP64 accumulation: dU^{n+1} = dU^n + (double)[2/3 ((dU^(2) - dU^n) + dt L)]
      float mnew[4];
      for (int v = 0; v < 4; v++) {
        const long long o = id + v * P;
        const float inc = (2.f / 3.f) * ((ld_stage<PERSIST>(In + o) - Mn[o]) + dt * L[v]);
        const double dn = ld_stage<PERSIST>(D + o) + (double)inc;
        D[o] = dn;
        mnew[v] = (float)dn;
        Mn[o] = mnew[v];
      }
      if (fuse_cfl) lam = cfl_lambda(k, c, mnew);
    }
  } else if (!DUAL && BODY && STAGE == 3 && inside && mytag != SOLID) {
    // IB / ghost node: the mirror of U^{n+1} takes the value rebuilt at stage 1
    for (int v = 0; v < 4; v++) Mn[id + v * P] = (float)ld_stage<PERSIST>(D + id + v * P);
  }
  // one call site for the whole block (the reduction has a barrier)
  if (STAGE == 3 && fuse_cfl) cfl_block_max(k, lam, lred, ds, ncfl, PERSIST);
}


}  // namespace ibm
