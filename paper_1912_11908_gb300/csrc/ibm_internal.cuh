// Internal declarations of the sm_103a immersed-boundary library (not installed).
#pragma once

#include <cuda.h>  // CUtensorMap (types only; the encoder is looked up at run time)
#include <cuda_runtime.h>
#include <stdint.h>

#include "ibm.h"

namespace ibm {

constexpr int NG = 3;  // halo / ghost layers for the five-point WENO stencil (Sec. 5)
constexpr int STAGE_TILE = 16;  // stage kernels: square tiles of STAGE_TILE x STAGE_TILE cells

enum : uint8_t { FLUID = 0, SOLID = 1, IB = 2, G1 = 3, G2 = 4, G3 = 5 };

// device-resident per-case scalars
struct DevState {
  double t;                      // time at the start of the current step
  double dt;                     // step size of the current step (set by the CFL reduction)
  unsigned long long lmax_bits;  // max spectral radius (bits of a positive double); 0 between reductions
  unsigned int done;             // blocks of the CFL reduction that have finished; 0 between reductions
  float dtf;                     // dt rounded to FP32
  int nbody_tiles;               // FP32-bulk: tiles that rebuild IB / ghost nodes
  double tst[2];                 // FP32-bulk: times of stages 2 and 3 (written during stage 1)
  int count[4];                  // #IB, #G1, #G2, #G3
  int offset[5];                 // exclusive prefix of count; offset[4] = total
  int err;                       // bit 0: list capacity exceeded, bit 1: empty stencil
  int pad;
  double pos[2];                 // body displacement at the last classification
  double bbox[4];                // xmin, xmax, ymin, ymax of the current pose
  int bcell[4];                  // cell index range ilo, ihi, jlo, jhi of centres in bbox, widened by 3 cells
  int urect[4];                  // cells re-classified this step: bcell (clipped) united with prect
  int prect[4];                  // bcell (clipped) of the previous classification
  int prect_valid;               // 0 before the first classification
  double force[4];               // Cd, Cl, Fx, Fy
  long long steps;
  double dt_next;                // persistent step kernel: dt of the next step, applied when the step ends
  float dtf_next;
  int pad2;
  // body free to translate under the fluid force (Eq. 10): displacement, velocity and acceleration at bt, the
  // start of the current step, and the force that set the acceleration
  double bX[2], bV[2], bA[2], bF[2], bt;
  // surface force (Eq. 9): per-block partial sums of the force kernel and the blocks finished (0 between calls)
  double fpart[2 * 64];
  unsigned int fdone;
  int pad3;
};

// IB / ghost lists up to this capacity are rebuilt by a single 1024-thread
// block per stage (IB nodes, barrier, ghost nodes); larger lists use two
// launches.
constexpr int RECON_ONE_BLOCK_MAX = 1 << 16;

constexpr int ERR_CAPACITY = 1;
constexpr int ERR_STENCIL = 2;
constexpr int ERR_TIMEOUT = 4;  // a bounded device wait (TMA completion) gave up

// body motion (prescribed translation)
struct Motion {
  int kind;
  double amp[2], freq, vel[2];
  double mass;  // COUPLED: body mass per unit depth
  double pivot[2], pmean, pamp;  // PITCH: centre of rotation, mean incidence and amplitude
};

// everything a kernel needs about the grid and the gas, passed by value
struct Consts {
  int nx, ny, pitch, rows;
  long long plane;  // pitch * rows
  double x0, y0, dx, dy, h, dmin;
  double gamma, R, cp, mu, kappa, pinf, prandtl, cfl, dt_fixed, ref_len;
  double uinf[2];
  double Uinf[4];   // free-stream conserved state
  double Hinf;      // free-stream total enthalpy
  int bc[4];
  Motion motion;
  int dual;         // dual time stepping (preconditioned pseudo time, BDF2 physical time)
  int ib_advance;   // IB nodes advanced by the flux update; the ghost layers alone impose the wall
  int subiters;     // dual time: sub-iterations per physical step
  double dt_phys;   // dual time: physical step
  double cfl_tau;   // dual time: pseudo-time CFL number
  double iR, ig1;   // 1/R and 1/(gamma - 1)
  double idt_phys;  // dual time: 1/dt_phys
  int tvd2;         // face reconstruction: TVD-2 (MUSCL, minmod) instead of WENO5
  int quad;         // IB / ghost reconstruction: quadratic along the normal (IBM_INTERP_QUADRATIC)
};


// geometry arrays (device)
struct RStencilQ;
struct Geom {
  int nv;
  const double *vref;   // 2*nv reference vertices
  double *vx, *vy;      // current pose
  double *snx, *sny, *vnx, *vny;   // segment and vertex normals of the current pose
  const double *rsnx, *rsny, *rvnx, *rvny;  // PITCH: normals of the reference pose (rotated into snx ...)
  const double *vk;     // signed curvature at each vertex (convex > 0)
  float *sb;            // per segment of the current pose, FP32: centre x, y and bounding radius (the stencil
                        // searches' pruning bounds, written by the pose kernels)
  int stencil_lanes;    // lanes per listed node of the stencil searches (16 or 32, from the body's size)
  RStencilQ *rsq;       // FP32-bulk with IBM_INTERP_QUADRATIC: the quadratic part of the compact stencils (else
                        // null), written with them
};

// The FP32 bounding circle of the segment (ax, ay) - (bx, by): centre, and half length plus a margin of 1e-5 of
// the coordinates' size (far above FP32 rounding), so that FP32 distances to the centre bound the distance to
// the segment from below and above.
__device__ __forceinline__ void segment_bound(double ax, double ay, double bx, double by, float *out) {
  const double cx = 0.5 * (ax + bx), cy = 0.5 * (ay + by);
  const double hl = 0.5 * sqrt((bx - ax) * (bx - ax) + (by - ay) * (by - ay));
  out[0] = (float)cx;
  out[1] = (float)cy;
  out[2] = (float)(hl + 1e-5 * (1.0 + fabs(cx) + fabs(cy) + hl));
}

__host__ __device__ inline long long cidx(const Consts &k, int i, int j) {
  return (long long)(j + NG) * k.pitch + (i + NG);
}

// Domain halos, applied while a tile is loaded: maps a cell index outside
// [0, n) to the interior cell that feeds it (periodic or zero-gradient
// outflow), or returns false for a free-stream side.  A corner takes the free
// stream if either side is free stream.
__device__ __forceinline__ bool halo_axis(int bc_lo, int bc_hi, int n, int &i) {
  if (i >= 0 && i < n) return true;
  const int b = i < 0 ? bc_lo : bc_hi;
  if (b == IBM_BC_PERIODIC) {
    i = ((i % n) + n) % n;
    return true;
  }
  if (b == IBM_BC_OUTFLOW) {
    i = i < 0 ? 0 : n - 1;
    return true;
  }
  return false;
}

__device__ __forceinline__ bool halo_map(const Consts &k, int &i, int &j) {
  const bool ax = halo_axis(k.bc[0], k.bc[1], k.nx, i);
  const bool ay = halo_axis(k.bc[2], k.bc[3], k.ny, j);
  return ax && ay;
}

// stage times of SSP-RK3: t_k = t + c_k dt, c = (0, 1, 1/2)
__device__ __forceinline__ double stage_time(const DevState *ds, int stage) {
  const double dt = ds->dt;
  return stage == 1 ? ds->t : (stage == 2 ? ds->t + dt : ds->t + 0.5 * dt);
}

// Last block of a CFL reduction: turn the maximum spectral radius into dt and
// reset the reduction state for the next step.  Call from thread 0 after the
// block's atomicMax; nblocks = blocks taking part (of one or more kernels).
// defer: store dt as the next step's (dt_next), for a kernel that still reads
// the current dt.
__device__ __forceinline__ void finish_cfl(const Consts &k, DevState *ds, unsigned int nblocks, bool defer = false) {
  __threadfence();
  const unsigned int ticket = atomicAdd(&ds->done, 1u);
  if (ticket == nblocks - 1) {
    __threadfence();
    const unsigned long long bits = atomicAdd(&ds->lmax_bits, 0ull);
    const double dt = k.cfl / __longlong_as_double((long long)bits);
    if (defer) {
      ds->dt_next = dt;
      ds->dtf_next = (float)dt;
    } else {
      ds->dt = dt;
      ds->dtf = (float)dt;
    }
    ds->lmax_bits = 0ull;
    ds->done = 0u;
  }
}

// motion state at time t
__device__ inline void motion_at(const Motion &m, double t, double X[2], double V[2], double A[2]) {
  X[0] = X[1] = V[0] = V[1] = A[0] = A[1] = 0.0;
  if (m.kind == IBM_MOTION_SIN) {
    const double w = 2.0 * 3.14159265358979323846 * m.freq;
    double s, c;
    sincos(w * t, &s, &c);
    for (int d = 0; d < 2; d++) {
      X[d] = m.amp[d] * s;
      V[d] = m.amp[d] * w * c;
      A[d] = -m.amp[d] * w * w * s;
    }
  } else if (m.kind == IBM_MOTION_CONST) {
    for (int d = 0; d < 2; d++) {
      X[d] = m.vel[d] * t;
      V[d] = m.vel[d];
    }
  }
}

// Pitching (Sec. 7.2): body angle theta = -alpha(t) (counter-clockwise positive), its rate and acceleration.
__device__ inline void pitch_at(const Motion &m, double t, double *th, double *om, double *al) {
  const double w = 2.0 * 3.14159265358979323846 * m.freq;
  double s, c;
  sincos(w * t, &s, &c);
  *th = -(m.pmean - m.pamp * c);
  *om = -m.pamp * w * s;
  *al = -m.pamp * w * w * c;
}

// Wall velocity and acceleration at the surface point (px, py): the body's translation, plus for a pitching
// body the rigid rotation about the pivot, V = om x r and A = al x r - om^2 r (r from the pivot).
__device__ inline void wall_kin(const Consts &k, double t, double px, double py, const double V0[2],
                                const double A0[2], double V[2], double A[2]) {
  if (k.motion.kind != IBM_MOTION_PITCH) {
    V[0] = V0[0];
    V[1] = V0[1];
    A[0] = A0[0];
    A[1] = A0[1];
    return;
  }
  double th, om, al;
  pitch_at(k.motion, t, &th, &om, &al);
  const double rx = px - k.motion.pivot[0], ry = py - k.motion.pivot[1];
  V[0] = V0[0] - om * ry;
  V[1] = V0[1] + om * rx;
  A[0] = A0[0] - al * ry - om * om * rx;
  A[1] = A0[1] + al * rx - om * om * ry;
}

// Body motion at time t: the prescribed forms, or, for a body translating
// under the fluid force (Eq. 10), the constant-acceleration motion of the
// current step from its start bt.
__device__ inline void body_motion(const Consts &k, const DevState *ds, double t, double X[2], double V[2],
                                   double A[2]) {
  if (k.motion.kind == IBM_MOTION_COUPLED) {
    const double tau = t - ds->bt;
    for (int d = 0; d < 2; d++) {
      A[d] = ds->bA[d];
      V[d] = ds->bV[d] + tau * ds->bA[d];
      X[d] = ds->bX[d] + tau * ds->bV[d] + 0.5 * tau * tau * ds->bA[d];
    }
    return;
  }
  motion_at(k.motion, t, X, V, A);
}

// Eq. 7 holds for a moving body whose speed relative to the free stream
// exceeds the free-stream sound speed (c_inf^2 = gamma p_inf / rho_inf =
// gamma R in the nondimensional gas).
__device__ inline bool supersonic_motion(const Consts &k, const double V[2]) {
  if (k.motion.kind == IBM_MOTION_STATIC) return false;
  const double rx = V[0] - k.uinf[0], ry = V[1] - k.uinf[1];
  return rx * rx + ry * ry > k.gamma * k.R;
}

struct RStencil32;

// ---- launchers (geometry.cu) ----
void launch_normals(int nv, const double *v, double *snx, double *sny, double *vnx, double *vny, double *vk,
                    cudaStream_t s);
void launch_pose(const Consts &k, const Geom &g, DevState *ds, cudaStream_t s);
// maxw x maxh: upper bound (cells) of the body's bounding box for any pose
void launch_classify(const Consts &k, const Geom &g, uint8_t *solid, const DevState *ds, int maxw, int maxh,
                     cudaStream_t s);
void launch_tags(const Consts &k, const uint8_t *solid, uint8_t *tag, int *blockcounts, DevState *ds, int cap,
                 ibm_stencil *st, cudaStream_t s, int *nlaunch);
void launch_stencils(const Consts &k, const Geom &g, const uint8_t *tag, ibm_stencil *st, int cap, DevState *ds,
                     cudaStream_t s);
// Opt the fused geometry kernels into the shared memory they use (once per device; before any capture).
void prepare_geometry_kernels();
// Geometry of one classification for bodies of at most FUSED_MAX_VERTS
// vertices, restricted to the cells the body can occupy: (1) pose and
// ray-parity classification of the cells of the previous and current
// bounding-box rectangles, (2) one block: tags, row-major IB / G1-G3 lists,
// reset of the cell -> stencil map, body-tile flags and list, (3) stencils,
// with their compact FP32 form and the cell -> stencil map when rs != NULL.
// Invariant: outside the rectangle last processed every cell is fluid,
// untagged and unlisted (solid, tag and sid are cleared at creation).  Same
// results as the unrestricted kernels.  Returns the kernels launched.
constexpr int FUSED_MAX_VERTS = 1024;
// blockcounts: 4 ints per TAG_BLOCK cells of the grid (the multi-block lists of large bodies).  ss (with
// ev_tags): a side stream for the stencils, forked from s once the tags and lists are enqueued; the caller
// joins it to s before anything reads the stencils (null: everything on s).
int launch_fused_geometry(const Consts &k, const Geom &g, uint8_t *solid, uint8_t *tag, ibm_stencil *st, int cap,
                          RStencil32 *rs, int *sid, uint8_t *tile_body, int *body_tiles, int body_cap, int maxw,
                          int maxh, DevState *ds, int *blockcounts, cudaStream_t s, cudaStream_t ss = nullptr,
                          cudaEvent_t ev_tags = nullptr);
// A: FP64 state, absolute conserved (pert = false) or perturbation (pert = true)
void launch_body_end(DevState *ds, cudaStream_t s);
// surf (optional): per segment the pressure and skin-friction coefficients, surf[e] and surf[nv + e]
void launch_forces_f64(const Consts &k, const Geom &g, const uint8_t *tag, const double *A, bool pert,
                       DevState *ds, cudaStream_t s, bool set_accel = false, double *surf = nullptr);

// ---- launchers (flow.cu) ----
void launch_dt(const Consts &k, const double *A, const uint8_t *tag, DevState *ds, cudaStream_t s, int *nlaunch);
void launch_recon_f64(const Consts &k, double *U, const ibm_stencil *st, int cap, const DevState *ds,
                      int stage, cudaStream_t s, int *nlaunch);
void launch_stage_f64(const Consts &k, int stage, const double *Un, const double *In, double *Out,
                      const uint8_t *tag, DevState *ds, cudaStream_t s);
// dual time: one pseudo-time stage (RK3 stage 1..3) of a sub-iteration; Q0 = iterate at the sub-iteration
// start (held in A), Wn / Wm the states at time levels n and n-1
void launch_dual_f64(const Consts &k, int stage, const double *A, const double *In, double *Out, const double *Wn,
                     const double *Wm, const uint8_t *tag, DevState *ds, cudaStream_t s);
void launch_dual_end(const Consts &k, DevState *ds, cudaStream_t s);

// Compact FP32 form of an IB / ghost stencil for the FP32-bulk reconstruction
// (built once per classification from the FP64 record).
struct RStencil32 {
  int cell;     // state index of the node
  int corner;   // state index of corner (i0, j0)
  int mask;     // bits 0-3 valid corners, bit 4 set for an IB node (ghost otherwise)
  float ratio;  // xi_node / xi_probe
  float dxi;    // xi_probe - xi_node
  float nx, ny;
  int ccell;    // interior index j0*nx + i0 of corner (i0, j0)
  float w[4];
  float curv;   // signed surface curvature at P' (supersonic moving-body condition, Eq. 7)
  float rx, ry; // P' relative to the pivot of a pitching body (0 otherwise)
};

// The quadratic reconstruction's part of a node's FP32 stencil (IBM_INTERP_QUADRATIC; a second array beside
// the RStencil32 records, read only by the kernels compiled for that form): the second probe's square, and the
// weights of the quadratics in the distance s along the normal, with s_n the node and s1, s2 the probes
struct RStencilQ {
  int corner;   // state index of corner (i0b, j0b)
  int ccell;    // interior index j0b*nx + i0b
  int mask;     // valid corners of the second square (0: none; the node takes the linear form)
  float w[4];
  float L1, L2; // Lagrange weights of the probes (Dirichlet velocity): s_n (s_n - s2) / (s1 (s1 - s2)), ...
  float m;      // (s_n^2 - s1^2) / (s2^2 - s1^2): weight of the second probe in the zero-slope quadratic
  float dq;     // (s_n - s1) - (s2 - s1) m: the pressure's change per unit wall slope
};

// the RStencilQ of a stencil record (weights from its FP64 distances)
__device__ __forceinline__ RStencilQ quad_stencil(const Consts &k, const ibm_stencil &s) {
  RStencilQ q;
  q.mask = s.maskb;
  q.corner = s.maskb ? (int)cidx(k, s.i0b, s.j0b) : 0;
  q.ccell = s.maskb ? s.j0b * k.nx + s.i0b : 0;
  for (int c = 0; c < 4; c++) q.w[c] = (float)s.wb[c];
  q.L1 = q.L2 = q.m = q.dq = 0.f;
  if (s.maskb) {
    const double s1 = s.xi_probe, s2 = s.xi_probe2, sn = s.xi_node;
    const double m = (sn * sn - s1 * s1) / (s2 * s2 - s1 * s1);
    q.L1 = (float)(sn * (sn - s2) / (s1 * (s1 - s2)));
    q.L2 = (float)(sn * (sn - s1) / (s2 * (s2 - s1)));
    q.m = (float)m;
    q.dq = (float)((sn - s1) - (s2 - s1) * m);
  }
  return q;
}

// FP32-bulk path (flow32.cu).  The FP64 state D of this mode holds the
// perturbation dU from the free stream (same variables as the FP32 arrays).
// U ([4][ny][nx] absolute conserved, contiguous, on the device) into A's padded layout; with M (FP32-bulk) as
// the perturbation from the free stream and its FP32 mirror
void launch_set_state(const Consts &k, const double *U, double *A, float *M, cudaStream_t s);
void launch_pert_to_abs64(const Consts &k, const double *D, double *A, cudaStream_t s);
void launch_dt_f32(const Consts &k, const float *M, const uint8_t *tag, DevState *ds, cudaStream_t s, int *nlaunch);
void launch_compact_stencils(const Consts &k, const ibm_stencil *st, RStencil32 *rs, RStencilQ *rsq, int *sid,
                             int cap, const DevState *ds, cudaStream_t s);
// Tiles of the stage kernel whose cells or 3-cell halo hold IB / ghost nodes
// ("body tiles"): flag per tile and a compact list (capacity body_cap).
// has_body = false: no vertices (every tile plain; ds->bbox unused).
// (Cases with a body of at most FUSED_MAX_VERTS vertices build their tile
// lists inside launch_fused_geometry instead.)
void launch_tile_lists(const Consts &k, const uint8_t *tag, uint8_t *tile_body, int *body_tiles, int body_cap,
                       DevState *ds, bool has_body, cudaStream_t s);
int stage_tiles(const Consts &k);
struct PertConsts {  // FP32 copies of the free-stream constants
  float gamma, g1, gg, R, Hinf, ux, uy, mu, kappa, idx, idy, dmin, vis, cp;
  float cfl_tau, idt_phys;  // dual time: pseudo-time CFL number, 1 / physical dt
};

__host__ inline PertConsts pert_consts(const Consts &k) {
  PertConsts c;
  c.gamma = (float)k.gamma;
  c.g1 = (float)(k.gamma - 1.0);
  c.gg = (float)(k.gamma / (k.gamma - 1.0));
  c.R = (float)k.R;
  c.Hinf = (float)k.Hinf;
  c.ux = (float)k.uinf[0];
  c.uy = (float)k.uinf[1];
  c.mu = (float)k.mu;
  c.kappa = (float)k.kappa;
  c.idx = (float)(1.0 / k.dx);
  c.idy = (float)(1.0 / k.dy);
  c.dmin = (float)k.dmin;
  c.vis = (float)((2.0 * k.gamma * k.mu / k.prandtl) * (1.0 / (k.dx * k.dx) + 1.0 / (k.dy * k.dy)));
  c.cp = (float)k.cp;
  c.cfl_tau = (float)k.cfl_tau;
  c.idt_phys = (float)k.idt_phys;
  return c;
}


// One FP32-bulk case of a stage batch: everything its stage kernels take.
// fuse_cfl: stage 3 also reduces the CFL maximum of the new state and sets the
// next step's dt (static bodies: the fluid set does not change between steps).
// Stage kernels of one case: the plain kernel (stream s) covers tiles without
// IB / ghost nodes near them; the body kernel (stream sb, may run concurrently)
// covers the listed body tiles and rebuilds IB and ghost nodes from rs / sid
// while it loads a tile (no separate reconstruction launch).  plain_variant
// selects the plain kernel's register budget, i.e. its resident blocks per SM
// (0: compiler's choice, 40 registers, six blocks; 1: 48 registers, five
// blocks; 2: about 60 registers, four blocks); with_body = false launches the
// plain kernel only (autotuning).
constexpr int PLAIN_VARIANTS = 3;
void launch_stage_f32(const Consts &k, int stage, float *Mn, const float *In, float *Out, double *D,
                      const uint8_t *tag, const int *sid, const RStencil32 *rs, const uint8_t *tile_body,
                      const int *body_tiles, int body_cap, DevState *ds, bool fuse_cfl, cudaStream_t s,
                      cudaStream_t sb, int plain_variant, bool with_body, const CUtensorMap *tmap,
                      const RStencilQ *rsq = nullptr);
// The same stage as one launch on stream s: body-tile slots first, then one
// block per tile (no second stream); pdl: launch with programmatic dependent
// launch, so that the launch overlaps the tail of the preceding stage kernel.
cudaError_t launch_stage_f32_one(const Consts &k, int stage, float *Mn, const float *In, float *Out, double *D,
                                 const uint8_t *tag, const int *sid, const RStencil32 *rs, const uint8_t *tile_body,
                                 const int *body_tiles, int body_cap, DevState *ds, bool fuse_cfl, int plain_variant,
                                 const CUtensorMap *tmap, bool pdl, cudaStream_t s,
                                 const RStencilQ *rsq = nullptr);
// Tensor maps of the FP32 stage inputs arrays[0..2] (pitch x rows x 4 planes)
// for the TMA staging of interior tiles (tmap above); false if the driver
// offers no encoder or the grid is too small for a box.
bool make_stage_tmaps(const Consts &k, float *const arrays[3], CUtensorMap out[3]);
// Persistent step kernel (step32.cu): the three SSP-RK3 stages of one
// explicit FP32-bulk step in one launch.  Blocks take (stage, tile) items in
// order from one counter: per stage the body tiles first (list order), then
// the other tiles (row-major); the item of stage s > 1 first waits until
// every tile within two tile columns and rows (wrapping across periodic
// sides) has finished stage s - 1.  Completion counts are epoch-based (3 x
// launches before + stages done), so only the claim counter is reset between
// launches; the last block to leave ends the step (t += dt, step count, next
// dt of the fused CFL) and rearms it.
struct StepSched {
  unsigned int next;    // next item to hand out
  unsigned int exited;  // blocks that have left the item loop
  unsigned int epoch;   // launches completed
  unsigned int pad;
  // followed by one completion count per tile
};
constexpr int STEP_VARIANTS = 2;  // register budget: 0 -> 40 registers (six blocks per SM), 1 -> 48 (five)
size_t step_sched_bytes(const Consts &k);
// grid of the persistent kernel: resident blocks per SM x SMs, at most 3 x tiles
int step_f32_grid(const Consts &k, int variant);
// tmaps: tensor maps of M, F1, F2 (NULL: per-thread tile loads)
cudaError_t launch_step_f32(const Consts &k, float *M, float *F1, float *F2, double *D, const uint8_t *tag,
                            const int *sid, const RStencil32 *rs, const uint8_t *tile_body, const int *body_tiles,
                            int body_cap, DevState *ds, StepSched *sch, bool fuse_cfl, const CUtensorMap *tmaps,
                            int variant, int grid, int s_first, int s_last, cudaStream_t s);
// Dual-time pseudo stage (1..3) in FP32-bulk form: residual of the FP32
// mirror In32, FP64 point-implicit update of the iterate In64 into Out64 (and
// its mirror Out32); D holds the sub-iteration's starting iterate, G the
// physical step's constant part of the BDF term (launch_dual_levels; all FP64
// perturbations); stage 1 stores the starting iterate's primitives in Q0 for
// stages 2 and 3.  Body tiles on sb.
void launch_dual_f32(const Consts &k, int stage, const float *In32, float *Out32, double *D, const double *In64,
                     double *Out64, const double *G, double *Q0, const uint8_t *tag, const int *sid,
                     const RStencil32 *rs, const uint8_t *tile_body, const int *body_tiles, int body_cap,
                     DevState *ds, cudaStream_t s, cudaStream_t sb, const RStencilQ *rsq = nullptr);
// Self-check of the dual update's integer-bit FP32 <-> FP64 conversions
// against the hardware conversions (synchronous, default stream).
cudaError_t check_float_conversions(unsigned long long *checked, unsigned long long *mismatched);
// Start of a physical step of FP32-bulk dual time: W^n <- A and, from the
// previous W^n (W^{n-1} of the new step), G = (W^{n-1} - 4 W^n) / (2 dt)
// (BDF2), or G = -W^n / dt on the first step (BDF1), over the whole padded
// state (4 planes).
void launch_dual_levels(const Consts &k, const double *A, double *Wn, double *G, const DevState *ds, cudaStream_t s);
// The same pseudo stage of a case with TVD-2 or the quadratic reconstruction
// as one launch on stream s (body-tile slots first); pdl: chained to the
// previous launch by programmatic dependent launch; rsq: the quadratic part
// of the compact stencils (required with the quadratic form).  (Other cases
// take launch_dual_f32_batch_one with a table of one.)
cudaError_t launch_dual_f32_var(const Consts &k, int stage, const float *In32, float *Out32, double *D,
                                const double *In64, double *Out64, const double *G, double *Q0,
                                const uint8_t *tag, const int *sid, const RStencil32 *rs, const uint8_t *tile_body,
                                const int *body_tiles, int body_cap, DevState *ds, bool pdl, cudaStream_t s,
                                const RStencilQ *rsq = nullptr);
// One member case of a group's block table (the request loop's batched
// stages: body-tile entries rebuild IB and ghost nodes from rs / sid while
// they load a tile, plain-tile entries cover the other tiles).
struct StageCase {
  Consts k;
  PertConsts c;
  float *M, *F1, *F2;  // mirror of U^n and the stage arrays
  double *D;           // FP64 master (perturbation)
  const uint8_t *tag;
  const int *sid;
  const RStencil32 *rs;
  const uint8_t *tile_body;
  const int *body_tiles;
  DevState *ds;
  int nt, nb;          // stage tiles, body-tile slots
  int fuse_cfl;
  unsigned int ncfl;   // blocks of the fused CFL reduction (nt + nb)
  // dual time only (null otherwise): the FP64 pseudo-stage iterates (D -> B -> C -> D), the BDF part of the
  // physical step and the sub-iteration's start primitives
  double *B, *C;
  const double *G;
  double *Q0;
  const RStencilQ *rsq;  // quadratic reconstruction: the quadratic part of the compact stencils (else null)
};

// Block table of a batched stage launch over the member cases of a group,
// passed by value in kernel parameter space: case q owns plain entries
// [plain_start[q], plain_start[q+1]) and body entries [body_start[q],
// body_start[q+1]).
constexpr int MAX_BATCH = 24;
struct StageBatch {
  int n;
  int plain_start[MAX_BATCH + 1];
  int body_start[MAX_BATCH + 1];
  StageCase cs[MAX_BATCH];
};
static_assert(sizeof(StageBatch) <= 32000, "kernel parameter space");
// fill b from n <= MAX_BATCH case descriptors
void build_stage_batch(const StageCase *cases, int n, StageBatch *b);

void fill_stage_case(const Consts &k, float *M, float *F1, float *F2, double *D, const uint8_t *tag, const int *sid,
                     const RStencil32 *rs, const uint8_t *tile_body, const int *body_tiles, int body_cap,
                     DevState *ds, bool fuse_cfl, StageCase *out);
// Stage `stage` of every case of the table as one launch over the combined
// table (body-tile entries first).  grid: blocks of the launch (<= 0 or >= the
// entries: one block per entry; fewer: persistent blocks striding over the
// table); pdl: chained to the previous launch by programmatic dependent launch.
cudaError_t launch_stage_f32_batch_one(const StageBatch &b, int stage, int grid, bool pdl, cudaStream_t s);
// Dual-time pseudo stage `stage` of every (dual-time, not TVD-2) case of the
// table as one launch over the combined table, with the same grid and pdl
// meanings: the one-launch form of a dual-time case alone (a table of one) and
// of a group of them.
cudaError_t launch_dual_f32_batch_one(const StageBatch &b, int stage, int grid, bool pdl, cudaStream_t s);

// ---- batching support (capi.cu), used by the request loop (serve.cu) ----
// FP32-bulk cases (explicit RK3 with any motion and either reconstruction,
// or dual time with WENO5 and the linear reconstruction) advance through
// batched stage launches.
bool case_batchable(const ibm_case *c);
// sub-iterations per physical step of a dual-time case (0: explicit RK3)
int case_subiters(const ibm_case *c);
// the stage kernels' variant a case needs: bit 0 TVD-2, bit 1 quadratic reconstruction (a group holds one)
int case_variant(const ibm_case *c);
// the case's body moves under the fluid force (Eq. 10)
bool case_coupled(const ibm_case *c);
// Work that must precede batched steps, on the case stream: the first
// classification and, for the fused CFL rule, the first dt (as ibm_step does
// outside its graph).
ibm_status case_prepare_batch(ibm_case *c);
// Per-step work before the stages, on the case stream: re-classification and
// stencils of a moving body; for a body under the fluid force, the force and
// the body's acceleration (Eq. 10); dt unless stage 3 provides it; for dual
// time, the rotation of the time levels.  Returns the kernels enqueued (0:
// nothing to do).  Graph-capturable.
int case_enqueue_prestage(ibm_case *c);
// Per-step work after the stages, on the case stream: the body update of
// Eq. 10, or the end of a dual-time physical step.  Returns the kernels
// enqueued.  Graph-capturable.
int case_enqueue_poststage(ibm_case *c);
void case_stage_desc(const ibm_case *c, StageCase *out);
cudaStream_t case_stream(const ibm_case *c);
void case_add_launches(ibm_case *c, long long n);

}  // namespace ibm
