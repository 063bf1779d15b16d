/*
 * ibm.h -- C ABI of the GB300 (sm_103a) sharp-interface immersed-boundary
 * compressible flow library.
 *
 * Method: Seshadri & De, arXiv 1912.11908.  One case is one 2-D uniform
 * Cartesian block with an immersed body given as a closed polyline.  Per
 * explicit time step the library runs, on the case's CUDA stream:
 *   - ray-casting classification of every cell centre and IB / ghost tagging
 *     (Sec. 3.2), for moving bodies at every step;
 *   - closest surface feature, pseudo-normal, boundary point and interpolation
 *     stencil of every IB and ghost node (Sec. 4.1-4.3, Eq. 1-3);
 *   - per Runge-Kutta stage: IB reconstruction (Sec. 4.4-4.6, Eq. 4-8), ghost
 *     field extension through image points into three layers (Sec. 5), domain
 *     halos, and the fused residual -- WENO5 reconstruction, low-diffusion flux
 *     splitting, central viscous flux -- with the stage update (Sec. 2);
 *   - surface force integration (Sec. 6, Eq. 9) on request.
 *
 * Conventions
 *   - Every call returns an ibm_status and never aborts; on error
 *     ibm_last_error() returns a thread-local message.
 *   - The library owns all device memory of a case.  Caller buffers passed to
 *     ibm_create_case are copied before it returns.
 *   - Work is enqueued on the stream given at creation; with NULL the case
 *     creates its own stream, which synchronises with the legacy default
 *     stream.  ibm_step is asynchronous; ibm_forces, ibm_get_state and
 *     ibm_sync synchronise that stream and report asynchronous device errors
 *     (list overflow -> IBM_ECAPACITY, empty interpolation stencil ->
 *     IBM_ESTENCIL, CUDA errors -> IBM_ECUDA).
 *   - Non-dimensionalisation: free-stream density 1 and temperature 1,
 *     reference speed 1, reference length 1; p_inf = 1/(gamma M^2),
 *     R = p_inf, mu = 1/Re (Re <= 0: inviscid), k = mu c_p / Pr.
 *   - Grid: nx * ny cells over [lo, hi]; cell (i, j) has centre
 *     (lo[0] + (i + 1/2) dx, lo[1] + (j + 1/2) dy).  Cell arrays exchanged with
 *     the caller are row-major [j][i] over the nx * ny interior cells.
 *   - A case is used by one host thread at a time.
 */
#ifndef IBM_GB300_H
#define IBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ibm_case ibm_case;

typedef enum {
  IBM_OK = 0,
  IBM_EINVAL = 1,     /* bad argument */
  IBM_ENOMEM = 2,     /* device allocation failed */
  IBM_ECAPACITY = 3,  /* more IB / ghost nodes than the case's list capacity */
  IBM_ESTENCIL = 4,   /* an IB / ghost node found no valid interpolation corner */
  IBM_ECUDA = 5,      /* CUDA runtime error */
  IBM_ESTATE = 6      /* call not valid in the case's current state */
} ibm_status;

/* node tags (Sec. 3.2, Sec. 5): fluid, solid, IB (fluid node with a solid
 * 4-neighbour), ghost layers G1..G3 (solid nodes whose nearest non-solid node
 * along a grid line is 1, 2 or 3 cells away) */
enum { IBM_TAG_FLUID = 0, IBM_TAG_SOLID = 1, IBM_TAG_IB = 2, IBM_TAG_G1 = 3, IBM_TAG_G2 = 4, IBM_TAG_G3 = 5 };
/* domain sides, in ibm_grid.bc order: x-low, x-high, y-low, y-high */
enum { IBM_BC_FREESTREAM = 0, IBM_BC_OUTFLOW = 1, IBM_BC_PERIODIC = 2 };
/* body motion: prescribed displacement X(t) = amp sin(2 pi freq t) (SIN) or vel t (CONST), or translation
 * under the fluid force (COUPLED, Sec. 6, Eq. 10): initial velocity vel, mass per unit depth `mass`; each step
 * the force at its start sets a constant acceleration F / mass for the step, the position advances by
 * U dt + dt^2 F / (2 mass) and the velocity by dt F / mass (explicit RK3 only), or pitching about a pivot
 * (PITCH, Sec. 7.2): incidence alpha(t) = pitch_mean - pitch_amp cos(2 pi freq t), nose up = clockwise, so the
 * body (given at zero incidence) is turned by -alpha(t) about `pivot`, its normals with it; the wall's velocity
 * and acceleration at a surface point r from the pivot are those of the rigid rotation, omega x r and
 * domega/dt x r - omega^2 r */
enum { IBM_MOTION_STATIC = 0, IBM_MOTION_SIN = 1, IBM_MOTION_CONST = 2, IBM_MOTION_COUPLED = 3, IBM_MOTION_PITCH = 4 };
/* arithmetic: FP64 throughout, or FP32 bulk (stage values and fluxes in FP32
 * on perturbations from the free stream, FP64 state accumulation) */
enum { IBM_PREC_FP64 = 0, IBM_PREC_FP32_BULK = 1 };
/* IB nodes (ibm_flow.ib_mode): rebuilt every stage, or advanced by the flux update */
enum { IBM_IB_REBUILD = 0, IBM_IB_ADVANCE = 1 };
/* time stepping: explicit SSP-RK3 with the CFL rule, or dual time (Sec. 2):
 * three-point (BDF2) physical-time derivative, preconditioned pseudo time,
 * each sub-iteration one point-implicit three-stage pseudo step with a 4x4
 * FP64 solve per cell; low-Mach scaling with the reference velocity
 * Ur = min(c, max(|V|, U_ref, nu/dx)) */
enum { IBM_TIME_RK3 = 0, IBM_TIME_DUAL = 1 };
/* face reconstruction of the inviscid flux (Sec. 2): fifth-order WENO (Jiang-Shu), or the second-order TVD
 * scheme read as MUSCL with the minmod limiter, f_i + 1/2 minmod(f_i - f_{i-1}, f_{i+1} - f_i), on the same
 * variables (rho, u, v, p) */
enum { IBM_SCHEME_WENO5 = 0, IBM_SCHEME_TVD2 = 1 };
/* IB and ghost reconstruction along the local normal n (distance s from the boundary point P'):
 *   LINEAR (default; the compressible form, Sec. 4.6 and Sec. 5): the velocity linear through the wall value and
 *     the probe (IB node) or mirror image point (ghost node), the temperature the probe's (adiabatic, Eq. 8), the
 *     pressure integrated from the probe under dp/dn = rho G with T fixed (Eq. 5-7);
 *   QUADRATIC (the incompressible form, Sec. 4.5 and Sec. 5): a second probe one diagonal spacing beyond the first
 *     (ibm_stencil *b fields) and quadratics in s through the wall condition and both probes -- Dirichlet velocity
 *     (Eq. 4), zero wall slope for the temperature, wall slope rho G for the pressure with the first probe's
 *     density -- evaluated at the node (s < 0 for a ghost node: extrapolation).  For smooth low-speed flow; the
 *     paper keeps the linear form wherever shocks can reach the wall. */
enum { IBM_INTERP_LINEAR = 0, IBM_INTERP_QUADRATIC = 1 };
/* stencil regions (Sec. 4.1): closest feature is a segment interior or a
 * vertex; FALLBACK = the line along the local normal met no segment on the
 * surface side, the boundary point is the closest point */
enum { IBM_REGION_FACE = 0, IBM_REGION_VERTEX = 1, IBM_REGION_FALLBACK = 2 };

/* Body: closed counter-clockwise polyline (interior on the left), nverts >= 3,
 * verts = 2*nverts doubles (x0, y0, x1, y1, ...), host memory, copied.  dim
 * must be 2. */
typedef struct {
  int dim;
  int nverts;
  const double *verts;
} ibm_geometry;

typedef struct {
  int nx, ny;       /* cells, each >= 8 */
  double lo[2], hi[2];
  int bc[4];        /* IBM_BC_* per side */
} ibm_grid;

typedef struct {
  double mach, re, gamma, prandtl, cfl;
  double uinf[2];   /* free-stream velocity in reference-speed units */
  double dt_fixed;  /* > 0: fixed time step, else the CFL rule (explicit scheme) */
  double ref_len;   /* force normalisation length (> 0) */
  int precision;    /* IBM_PREC_* */
  int time_scheme;  /* IBM_TIME_* */
  int subiters;     /* dual time: pseudo-time sub-iterations per physical step (>= 1) */
  int ib_mode;      /* IBM_IB_REBUILD: IB nodes rebuilt from their probes every stage (Sec. 4.4-4.6);
                       IBM_IB_ADVANCE: IB nodes advanced by the flux update, the wall imposed by the ghost
                       layers alone (Sec. 5) */
  double dt_phys;   /* dual time: physical time step (> 0) */
  double cfl_tau;   /* dual time: pseudo-time CFL number (> 0) */
  int scheme;       /* IBM_SCHEME_* */
  int ib_interp;    /* IBM_INTERP_* */
} ibm_flow;

typedef struct {
  int kind;         /* IBM_MOTION_* */
  double amp[2];
  double freq;
  double vel[2];    /* CONST: velocity; COUPLED: initial velocity */
  double mass;      /* COUPLED: body mass per unit depth (> 0), in units of rho_inf L^2 */
  double pivot[2];  /* PITCH: centre of rotation */
  double pitch_mean, pitch_amp;  /* PITCH: mean incidence and amplitude (radians) */
} ibm_motion;

/* One IB or ghost node and its reconstruction stencil (Sec. 4.1-4.6, Sec. 5).
 * The node value is rebuilt on the line P' + xi n through the boundary point
 * P' along the local normal n (face normal or vertex pseudo-normal, pointing
 * into the fluid); the probe (IB node) or image point (ghost node) sits at
 * xi_probe, the node at xi_node. */
typedef struct {
  int32_t cell;     /* j*nx + i */
  int32_t feature;  /* segment (FACE) or vertex (VERTEX) index */
  int32_t region;   /* IBM_REGION_* */
  int32_t i0, j0;   /* lower-left cell of the interpolation square */
  int32_t mask;     /* bit k set: corner k = (i0 + (k&1), j0 + (k>>1)) is valid */
  int32_t nstep;    /* probe push-outs (0..3) */
  int32_t kind;     /* 0 IB, 1..3 ghost layer */
  double nx, ny;    /* local normal */
  double bx, by;    /* boundary point P' */
  double xi_node, xi_probe;
  double w[4];      /* interpolation weights, 0 on invalid corners */
  double curv;      /* signed curvature 1/R of the surface at P' (convex > 0): linear along the segment holding
                       P' between the end vertices' Menger curvatures (Eq. 7, supersonic moving bodies) */
  /* IBM_INTERP_QUADRATIC: the second probe / image point, at xi_probe2 = xi_probe + one diagonal spacing (pushed
   * out like the first while its square has no valid corner), its square and weights; all zero otherwise or when
   * none was found (the node then takes the linear form) */
  int32_t i0b, j0b, maskb, nstepb;
  double xi_probe2;
  double wb[4];
} ibm_stencil;

/* what for ibm_get_state */
enum {
  IBM_STATE_FP64 = 0,   /* double[4][ny][nx]: rho, rho u, rho v, rho E */
  IBM_TAGS = 1,         /* uint8_t[ny][nx] */
  IBM_LIST_COUNTS = 2,  /* int32_t[4]: #IB, #G1, #G2, #G3 */
  IBM_STENCILS = 3,     /* ibm_stencil[#IB + #G1 + #G2 + #G3], IB first then G1, G2, G3, each in row-major order */
  IBM_TIME = 4,         /* double[2]: t, last dt */
  IBM_STEPS = 5,        /* int64_t: steps taken */
  IBM_TUNING = 6,       /* int32_t[2] (host only): register-budget variants of the FP32-bulk stage kernel
                           picked by the autotuner for stage 1 and for stages 2-3 (0..2; -1 before the first
                           step, or FP64) */
  IBM_STAGE_LAUNCH = 7, /* int32_t (host only): launch form of the FP32-bulk stages (0..2, see
                           ibm_stage_launches; the autotuner's pick unless set; -1 for FP64) */
  IBM_BODY = 8          /* double[6]: body displacement x, y and velocity u, v at the current time, and the
                           force per unit depth Fx, Fy that set the last step's acceleration (COUPLED; zeros
                           otherwise) */
};

/* Create a case, initialised to the uniform free stream at t = 0 (no
 * classification yet).  cuda_stream: a cudaStream_t or NULL.  motion may be
 * NULL (static body).  geometry->nverts may be 0 (no body). */
ibm_status ibm_create_case(const ibm_geometry *geometry, const ibm_grid *grid, const ibm_flow *flow,
                           const ibm_motion *motion, void *cuda_stream, ibm_case **out);

/* Classify cells, build IB / ghost lists and stencils at the current time
 * (Sec. 3.2, 4.1-4.3).  Asynchronous. */
ibm_status ibm_classify(ibm_case *c);

/* Advance nsteps physical steps (SSP-RK3, or dual time with `subiters`
 * sub-iterations).  Moving bodies are re-classified at the start of every
 * step; a static body is classified once if it has not been.  Asynchronous. */
ibm_status ibm_step(ibm_case *c, int nsteps);

/* Copy a quantity out.  dst: host memory (dst_on_device = 0) or device memory
 * on the case's device (1); bytes must be at least the size documented for
 * `what`.  Synchronises the case stream. */
ibm_status ibm_get_state(ibm_case *c, int what, void *dst, size_t bytes, int dst_on_device);

/* Overwrite the conserved state (double[4][ny][nx], as IBM_STATE_FP64) from
 * host or device memory.  Asynchronous for device sources; a host source is
 * copied before the call returns. */
ibm_status ibm_set_state(ibm_case *c, const void *src, size_t bytes, int src_on_device);

/* As ibm_set_state, asynchronous for host sources too: the copy is enqueued
 * on the case stream and the caller keeps src unchanged (and, for a host
 * source, page-locked if it wants the copy to overlap) until the next
 * synchronising call (ibm_forces, ibm_get_state, ibm_sync).  Lets a caller
 * upload, step and read forces with one host synchronisation per step. */
ibm_status ibm_set_state_async(ibm_case *c, const void *src, size_t bytes, int src_on_device);

/* Surface force at the current time (Sec. 6, Eq. 9): out = {Cd, Cl, Fx, Fy}
 * with C = F / (1/2 rho_inf U_ref^2 ref_len).  Synchronises. */
ibm_status ibm_forces(ibm_case *c, double out[4]);

/* Surface distributions at the current time (Sec. 6, the integrand of Eq. 9): for each of the body's nseg
 * segments (segment e runs from vertex e to vertex e + 1 of the current pose) the wall pressure coefficient
 * cp[e] = (p_s - p_inf) / (rho_inf U_ref^2 / 2) and the skin-friction coefficient cf[e] = tau_w /
 * (rho_inf U_ref^2 / 2) at its midpoint, evaluated exactly as ibm_forces evaluates them (p_s the probe
 * pressure carried to the wall by the wall condition, tau_w = mu (u_P - U_wall).t / h); NaN where no probe
 * square was found.  cp, cf: host arrays of nseg doubles (caller-owned).  IBM_EINVAL unless nseg equals the
 * body's vertex count.  Synchronises. */
ibm_status ibm_surface(ibm_case *c, double *cp, double *cf, int nseg);

/* ---- 3-D immersed-boundary pre-processing (Sec. 3.2, Sec. 4.1-4.2; Appendix A) ----
 *
 * A closed, consistently oriented triangulated surface (each directed edge in
 * one face, its reverse in the neighbouring face; counter-clockwise seen from
 * outside) against a uniform lattice of nx * ny * nz nodes over [lo, hi]: node
 * (i, j, k) sits at lo + (index + 1/2) (hi - lo) / n along each axis, node
 * index (k ny + j) nx + i.  One classification runs, on the body's stream:
 *   - ray casting (Sec. 3.2): nodes outside the surface's axis-aligned
 *     bounding box are fluid; inside it, rays along +x, +y and +z each count
 *     their crossings with the Moller-Trumbore barycentric test, written as
 *     the three edge functions of the face projected along the ray, every edge
 *     evaluated with its endpoints in increasing vertex index and a zero value
 *     resolved by a symbolic shift of the node, so that a crossing through an
 *     edge or a vertex counts exactly once; a node is solid when at least two
 *     of the three crossing counts are odd;
 *   - tagging over the 6-neighbourhood: IB = fluid node with a solid
 *     neighbour; G1..G3 = solid node whose nearest non-solid node along a
 *     lattice line is 1..3 nodes away (IBM_TAG_*);
 *   - ordered lists: the IB nodes, then G1, G2, G3, each in node-index order;
 *   - closest feature of every listed node (Sec. 4.1): exhaustive over the
 *     faces, the plane projection when it falls inside a face, else the
 *     nearest point of its edges; equal distances keep the lowest face; and
 *     its pseudo-normal (Sec. 4.2): the face normal, the angle-weighted vertex
 *     normal (Eq. 2) or the normalised sum of the two faces' normals at an edge
 *     (Eq. 3), all pointing out of the body.
 * The computation uses IEEE basic operations and sqrt only (face and vertex
 * normals, which need acos, are formed once on the host at creation), so its
 * results are reproducible bit for bit.  The 3-D flow solver (ibm_case3d_*
 * below) runs on these results. */
typedef struct ibm_body3d ibm_body3d;

typedef struct {
  int nx, ny, nz;   /* lattice nodes per axis, each >= 1, product < 2^31 */
  double lo[3], hi[3];
} ibm_grid3d;

enum { IBM_FEATURE_FACE = 0, IBM_FEATURE_EDGE = 1, IBM_FEATURE_VERTEX = 2 };

/* one listed node and its closest surface feature */
typedef struct {
  int32_t node;      /* node index (k ny + j) nx + i */
  int32_t tri;       /* face holding the closest point */
  int32_t kind;      /* IBM_FEATURE_* */
  int32_t reserved;
  double cp[3];      /* closest point on the surface */
  double n[3];       /* unit pseudo-normal of the feature, out of the body */
} ibm_closest3d;

/* what for ibm_body3d_get */
enum {
  IBM_3D_TAGS = 0,     /* uint8_t[nz][ny][nx] */
  IBM_3D_COUNTS = 1,   /* int32_t[4]: #IB, #G1, #G2, #G3 */
  IBM_3D_NODES = 2,    /* int32_t[#IB + #G1 + #G2 + #G3]: node indices, IB first, each class in index order */
  IBM_3D_CLOSEST = 3   /* ibm_closest3d[#IB + #G1 + #G2 + #G3], in the order of IBM_3D_NODES */
};

/* Copy a surface (verts: 3*nverts doubles, tris: 3*ntris vertex indices; host
 * memory, copied) to the device and form its face normals, angle-weighted
 * vertex normals and edge neighbours.  cuda_stream: a cudaStream_t or NULL
 * (the body then creates its own).  IBM_EINVAL for fewer than 4 vertices or
 * faces or an index out of range, IBM_ENOMEM / IBM_ECUDA on device errors. */
ibm_status ibm_body3d_create(const double *verts, int nverts, const int32_t *tris, int ntris, void *cuda_stream,
                             ibm_body3d **out);

/* Classify the lattice, tag it, build the lists and the closest features
 * (five kernels, asynchronous on the body's stream).  Device buffers are
 * (re)allocated when the lattice size changes; the lists hold the nodes
 * within three nodes of the bounding box.  IBM_EINVAL for an empty or
 * oversized lattice. */
ibm_status ibm_body3d_classify(ibm_body3d *b, const ibm_grid3d *grid);

/* Copy a result of the last classification to host memory (synchronises the
 * body's stream).  IBM_ESTATE before any classification; IBM_ECAPACITY (after
 * copying what fits) if the lists overflowed. */
ibm_status ibm_body3d_get(ibm_body3d *b, int what, void *dst, size_t bytes);

/* Release the body's device memory (and its own stream).  NULL is a no-op. */
ibm_status ibm_body3d_destroy(ibm_body3d *b);

/* ---- 3-D flow (Sec. 2-6 on a 3-D block; Appendix A's sphere) ----
 *
 * One uniform block of nx * ny * nz cells (cell (i, j, k) centred at lo +
 * (index + 1/2) (hi - lo) / n, index (k ny + j) nx + i) around a static closed
 * triangulated body (as for ibm_body3d_create; none when ntris = 0), in FP64,
 * advanced by explicit SSP-RK3 steps with the CFL rule (or dt_fixed).  At
 * creation the body is classified, tagged and listed on the lattice of cell
 * centres (ibm_body3d_classify) and every listed node gets its stencil:
 *   - the boundary point P' is the foot of the node X on the plane through its
 *     closest surface point C normal to the local normal n (the pseudo-normal
 *     of the closest feature, out of the body): P' = X - xi_node n with
 *     xi_node = (X - C).n -- the closest point itself on a face;
 *   - an IB node's probe lies one cell diagonal sqrt(dx^2 + dy^2 + dz^2)
 *     beyond the node along n; a ghost node's image point is its mirror image
 *     through P' (at least min(dx, dy, dz) / 2 from P'); either is pushed out
 *     by min(dx, dy, dz), up to three times, while its cube has no valid
 *     corner (IBM_ESTENCIL when none is found);
 *   - interpolation over the cube of the eight surrounding cell centres:
 *     trilinear when all eight are valid (fluid; fluid or IB for image
 *     points), else inverse-distance weights 1 / r^2 over the valid ones.
 * Per RK stage: IB nodes from their probes (static wall: velocity zero at P'
 * and linear along n, Eq. 4; pressure and temperature the probe's, Eq. 5-6
 * and 8), then the three ghost layers from their image points (Sec. 5), the
 * domain halos (free stream, zero-gradient outflow or periodic, as in 2-D),
 * and the fused residual of Sec. 2 in three directions -- WENO5 on (rho, u, v,
 * w, p), LDFSS(0), central viscous flux with the Stokes hypothesis -- with the
 * stage update of the fluid cells.  Forces follow Eq. 9 with one midpoint per
 * triangle, the probe one cell diagonal out along the face normal.  These
 * tags, lists and stencils are bit-identical to an FP64 evaluation of the same
 * formulas in IEEE basic operations; the FP64 state agrees with such an
 * evaluation to FP64 rounding. */
typedef struct ibm_case3d ibm_case3d;

typedef struct {
  int nx, ny, nz;   /* cells, each >= 4 */
  double lo[3], hi[3];
  int bc[6];        /* IBM_BC_* for x-low, x-high, y-low, y-high, z-low, z-high */
  double mach, re, gamma, prandtl, cfl;  /* re <= 0: inviscid */
  double uinf[3];   /* free-stream velocity in reference-speed units */
  double dt_fixed;  /* > 0: fixed time step, else the CFL rule */
  double ref_area;  /* force normalisation area (> 0) */
  int precision;    /* IBM_PREC_FP64, or IBM_PREC_FP32_BULK: stage values, IB / ghost reconstruction, halos, CFL
                       bound and fluxes in FP32 on perturbations from the free stream (rho - 1, u - U_inf,
                       p - p_inf, T - 1; the pressure flux less p_inf and the energy equation in rho E - rho H_inf,
                       so that no free-stream constant enters an FP32 sum), each step's increment accumulated onto
                       an FP64 master (the state that ibm_case3d_get returns and the forces read) */
} ibm_flow3d;

/* one IB or ghost node of the 3-D case and its stencil */
typedef struct {
  int32_t node;      /* (k ny + j) nx + i */
  int32_t kind;      /* 0 IB, 1..3 ghost layer */
  int32_t region;    /* closest feature: IBM_FEATURE_* */
  int32_t nstep;     /* probe push-outs (0..3) */
  int32_t i0, j0, k0;/* lowest corner of the interpolation cube */
  int32_t mask;      /* bit b set: corner (i0 + (b & 1), j0 + (b >> 1 & 1), k0 + (b >> 2)) valid */
  double n[3];       /* local normal */
  double b[3];       /* boundary point P' */
  double xi_node, xi_probe;
  double w[8];       /* interpolation weights, 0 on invalid corners */
} ibm_stencil3d;

/* what for ibm_case3d_get (IBM_3D_TAGS and IBM_3D_COUNTS as for ibm_body3d_get) */
enum {
  IBM_3D_STATE = 4,    /* double[5][nz][ny][nx]: rho, rho u, rho v, rho w, rho E */
  IBM_3D_STENCILS = 5, /* ibm_stencil3d[#IB + #G1 + #G2 + #G3], IB first, each class in node-index order */
  IBM_3D_TIME = 6      /* double[2]: t, last dt */
};

/* Create a case at the uniform free stream, t = 0, classify its body and build
 * the stencils (synchronous).  verts: 3*nverts doubles, tris: 3*ntris indices
 * (host, copied; ntris = 0: no body).  cuda_stream: a cudaStream_t or NULL
 * (the case then creates its own, which synchronises with the legacy default
 * stream).  IBM_EINVAL for bad arguments, IBM_ESTENCIL
 * if a listed node finds no probe corner, IBM_ENOMEM / IBM_ECUDA on device
 * errors (no case is returned then). */
ibm_status ibm_case3d_create(const double *verts, int nverts, const int32_t *tris, int ntris,
                             const ibm_flow3d *flow, void *cuda_stream, ibm_case3d **out);

/* Advance nsteps SSP-RK3 steps.  Asynchronous. */
ibm_status ibm_case3d_step(ibm_case3d *c, int nsteps);

/* Copy a quantity to host (dst_on_device = 0) or device memory (1); bytes at
 * least its size.  Synchronises the case stream. */
ibm_status ibm_case3d_get(ibm_case3d *c, int what, void *dst, size_t bytes, int dst_on_device);

/* Overwrite the conserved state (double[5][nz][ny][nx]) from host or device
 * memory (a host source is copied before the call returns). */
ibm_status ibm_case3d_set_state(ibm_case3d *c, const void *src, size_t bytes, int src_on_device);

/* Force on the body at the current state (Eq. 9): out = {Cx, Cy, Cz, Fx, Fy,
 * Fz}, C = F / (1/2 rho_inf U_ref^2 ref_area).  Synchronises. */
ibm_status ibm_case3d_forces(ibm_case3d *c, double out[6]);

/* Kernel launches enqueued by the case so far. */
int64_t ibm_case3d_launch_count(const ibm_case3d *c);

/* Release the case (synchronises first).  NULL is a no-op. */
ibm_status ibm_case3d_destroy(ibm_case3d *c);

/* Measured arithmetic ceiling (no counterpart in the paper; the rooflines of the ALU-bound kernels are
 * taken against it): one launch of iters fused multiply-adds per recurrence, 8 independent recurrences per
 * thread, 4 blocks of 256 threads per SM, in FP32 (fp64 = 0) or FP64 (fp64 = 1) on the current device,
 * after a short warm-up launch.  flops_per_s = 2 x FMAs / the launch's CUDA-event time, ms = that time.
 * Allocates and frees a small output buffer; synchronises the device's legacy default stream.
 * IBM_EINVAL for iters <= 0 or NULL outputs. */
ibm_status ibm_fma_peak(int fp64, long long iters, double *flops_per_s, double *ms);

/* Wait for the case's stream; report asynchronous errors. */
ibm_status ibm_sync(ibm_case *c);

/* Release every resource of the case (synchronises first).  NULL is a no-op. */
ibm_status ibm_destroy_case(ibm_case *c);

/* Device bytes held by a case of these sizes (admission control). */
size_t ibm_case_device_bytes(const ibm_geometry *geometry, const ibm_grid *grid, const ibm_flow *flow,
                             const ibm_motion *motion);

/* Kernel launches enqueued by the case so far (instrumentation; a step
 * replayed from a CUDA graph counts the kernels it contains). */
int64_t ibm_launch_count(const ibm_case *c);

/* Instrumentation.  While enabled, ibm_step launches kernels directly (no
 * graph replay) and records CUDA events on the case stream around each kernel
 * group; ibm_profile_read synchronises, writes per group the summed device
 * time in ms and the number of timed launches, and clears the record.
 * Groups: 0 fused residual + stage update, 1 IB / ghost reconstruction,
 * 2 domain halos, 3 time-step reduction, 4 geometry (pose, classification,
 * tags, lists, stencils), 5 end of step.  n_groups <= 6. */
ibm_status ibm_profile_enable(ibm_case *c, int enable);
ibm_status ibm_profile_read(ibm_case *c, double *ms, int64_t *launches, int n_groups);

/* Autotuning (default on).  FP32-bulk explicit cases time the stage kernels
 * (plain tiles and the concurrent body tiles) under three register budgets of
 * the plain kernel (six, five and four resident blocks per SM), separately
 * for stage 1 and stage 2, on their first ibm_step -- about a hundred extra
 * launches and a few host waits -- and keep the fastest (stage 3 follows
 * stage 2); the choice is cached per device and grid size for the process.  enable = 0 uses the compiler's default budget.  Results do not
 * depend on the choice beyond FP32 rounding.  Only before the first step
 * (IBM_ESTATE afterwards). */
ibm_status ibm_autotune(ibm_case *c, int enable);

/* FP32-bulk explicit stages: stage the loaded region (tile + 3-cell halo) of
 * every tile that needs no domain-halo mapping into shared memory with one TMA
 * tensor copy (cp.async.bulk.tensor) per tile instead of per-thread loads
 * (default on where the driver provides the tensor-map encoder).  The values
 * loaded are the same, so results do not depend on the choice.  enable = 0
 * uses per-thread loads for every tile.  The wait for a copy is bounded by
 * about a second of the GPU's global timer; a block whose copy has not
 * completed by then waits once more (bounded), leaves its tile unprocessed and
 * flags the case: the next synchronising call returns IBM_ECUDA and the
 * state of that step is invalid. */
ibm_status ibm_use_tma(ibm_case *c, int enable);

/* FP32-bulk stages (Sec. 2; explicit stages and dual-time pseudo stages): how
 * each stage is launched.
 *   0: a plain-tile kernel and a body-tile kernel on two streams;
 *   1: one kernel holding both, body-tile blocks first;
 *   2: as 1, each stage launched with programmatic dependent launch, so that
 *      its blocks are resident, waiting for the previous stage, while the
 *      previous stage's last blocks finish.
 * Unless this is called, the autotuner times forms 0 and 2 with their
 * register budgets on an explicit case's first step and keeps the faster
 * (IBM_STAGE_LAUNCH reports it; without autotuning, and for dual time, the
 * form is 2).  Modes 1 and 2 run the same
 * kernel and give bit-identical results; mode 0's kernels are compiled
 * separately (results agree to FP32 rounding).  IBM_EINVAL for another mode. */
ibm_status ibm_stage_launches(ibm_case *c, int mode);

/* FP32-bulk explicit steps: run the three SSP-RK3 stages of a step (Sec. 2)
 * as one persistent launch instead of one plain-tile and one body-tile launch
 * per stage (default off).  Blocks take (stage, tile) items in order; a
 * tile's next stage starts as soon as the tiles within two tiles of it have
 * finished the previous one, so stages overlap across the grid.  Each tile
 * runs the same arithmetic as in the per-stage launches (separately compiled:
 * results agree to FP32 rounding).  On GB300 it matches the per-stage
 * launches on grids of about one wave of tiles per stage and is slower on
 * larger ones.  A dependency wait that gives up (it cannot, short of a fault)
 * makes the next sync report IBM_ECUDA. */
ibm_status ibm_use_persistent(ibm_case *c, int enable);

/* Blocks of the persistent step kernel: 0 (default) = as many as are resident
 * at once on the device; a smaller number (at least 1; larger values are
 * clipped to the default) runs fewer items concurrently -- 1 runs every
 * (stage, tile) item in order on one block.  The result does not depend on
 * it. */
ibm_status ibm_persistent_grid(ibm_case *c, int blocks);

/* Self-check of the FP32 <-> FP64 conversions that the FP32-bulk dual-time
 * update (Sec. 2) performs on the integer bits of IEEE 754 values (off the
 * FP64 pipe, which bounds that update): on the current device, compares them
 * with the hardware conversions for every binary32 bit pattern except the
 * subnormals (which the FP32 arithmetic flushes to zero) and for 2^30
 * pseudo-random binary64 patterns, one in four an exact rounding tie, with
 * exponents from below to above the binary32 range.  *checked receives the
 * number of values compared, *mismatched those that differ in any bit (NaN
 * against NaN counts as equal); both host pointers.  Synchronous; takes about
 * a second.  IBM_EINVAL for a NULL pointer, IBM_ECUDA if a CUDA call fails. */
ibm_status ibm_check_float_conversions(uint64_t *checked, uint64_t *mismatched);

/* Replay each step from a CUDA graph captured on first use (default on);
 * enable = 0 launches every kernel directly. */
ibm_status ibm_use_graphs(ibm_case *c, int enable);

const char *ibm_last_error(void);

/* Allocation-free classification, tagging and list compaction.  (The paper
 * has no counterpart; this is a library facility.)
 *
 * For callers that cannot allocate device memory: code that runs where
 * cudaMalloc is unavailable or not allowed (a host callback, an embedding
 * that owns every device allocation, a memory pool that must not grow after
 * start-up).  It computes the same tags and the same row-major IB / G1 / G2 /
 * G3 lists as ibm_classify, for a body given at its current pose, without any
 * case and without allocating: its intermediate data lives in one fixed
 * device array inside the library (about 4.3 MiB, held on every GPU that
 * loads the library until the process exits).
 *
 * grid:     host struct (bc is ignored); nx * ny <= 4194304 cells.
 * d_verts:  device, 2*nverts doubles (x0, y0, x1, y1, ...), closed CCW
 *           polyline, 3 <= nverts <= 4096.
 * d_tags:   device output, uint8_t[ny][nx] (IBM_TAG_*).
 * d_cells:  device output, int32_t[capacity]: cell indices j*nx+i of the IB
 *           nodes, then G1, G2, G3, each in row-major order; entries past
 *           capacity are not written.
 * d_counts: device output, int32_t[4]: #IB, #G1, #G2, #G3 (full totals, even
 *           when they exceed capacity).
 * Asynchronous on cuda_stream (NULL = legacy default stream).  Sizes beyond
 * the limits return IBM_EINVAL before any GPU work.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.  The
 * address is kept for the life of the process: after cudaDeviceReset (or any
 * teardown of the device's primary context) it is stale, so do not call this
 * entry point on that device again in the same process.  All calls share the
 * one array, so calls that overlap on the GPU (other streams, other host
 * threads) race and must be serialised by the caller. */
ibm_status ibm_tag_nodes_noalloc(const ibm_grid *grid, const double *d_verts, int nverts, uint8_t *d_tags,
                                 int32_t *d_cells, int32_t capacity, int32_t *d_counts, void *cuda_stream);

/* Request loop (continuous batching of many cases on one GPU).  (The paper
 * solves one configuration at a time and has no counterpart; this is a
 * library facility built on the calls above.)
 *
 * A server queues solve requests -- body, grid, flow, motion and a number of
 * steps (explicit steps, or physical steps in dual time) -- and admits them in
 * arrival order while fewer than
 * max_active cases are running and the device bytes of the running cases
 * (ibm_case_device_bytes) plus the next request's stay within the budget.
 * Each admitted case owns its device state, tags and lists and a stream of
 * its own; it is classified once and advanced in chunks of steps_per_chunk
 * steps replayed from its CUDA graph, so the kernels of all running cases
 * overlap on the device.  A case that has taken all its steps is retired:
 * its forces and time are read, its device memory is freed and the slot
 * goes to the next waiting request.  Cases share nothing on the device, so
 * a request gives the same result alone and in any mix.
 *
 * Batched mode (default) for FP32-bulk requests (explicit RK3 with any
 * motion, including a body under the fluid force, and either reconstruction
 * and IB form; dual time with WENO5 and the linear IB form):
 * the requests admitted in one pass form groups of up to 24 cases of similar
 * size (grids within a factor four in cells), equal step counts, the same
 * time scheme (dual time: equal sub-iteration counts) and the same scheme and
 * IB form.  One step of a group is
 * one CUDA graph: the per-case work before the stages (re-classification of
 * moving bodies, the force and acceleration of Eq. 10, dt, or the rotation of
 * the dual-time levels) on the cases' streams; per RK stage, or per pseudo
 * stage of every sub-iteration, one launch over the block table of all member
 * cases; then the per-case work that ends the step (the body update of
 * Eq. 10, the end of a dual-time step).  A group's membership is fixed when it
 * forms (its graph is captured once and its members finish together); later
 * arrivals form new groups, which run beside the old ones.  With
 * IBM_SERVE_AUTOTUNE the stage launch's schedule of an explicit group whose
 * bodies do not move under the fluid force (one block per tile, or a
 * persistent grid striding over the table) is picked by timing the candidates
 * on the group, once per size class and membership size.  Other requests
 * (FP64; dual time with TVD-2 or the quadratic IB form), and all requests
 * when batching is off, advance on their own streams as described above.
 * Results do not depend on the mix; they are bit-identical to a case stepped alone on the own-stream path and, for
 * dual-time requests, in a group; explicit requests in a group are equal up
 * to FP32 rounding (the group's stage kernel is compiled separately).
 *
 * The server is driven by the caller's thread: ibm_server_progress does one
 * non-blocking pass (retire finished cases, admit waiting requests, enqueue
 * the next chunk of every case or group whose previous chunk is done).  Call
 * it in a loop until it reports no running and no waiting request.  One host
 * thread at a time per server; cases are created on the current device. */
typedef struct ibm_server ibm_server;

enum { IBM_REQ_PENDING = 0, IBM_REQ_RUNNING = 1, IBM_REQ_DONE = 2, IBM_REQ_FAILED = 3 };
enum { IBM_SERVE_BATCHED = 1, IBM_SERVE_AUTOTUNE = 2 };
#define IBM_SERVER_NSTATS 5

typedef struct {
  int64_t id;
  int32_t state;      /* IBM_REQ_* */
  int32_t status;     /* ibm_status of the request (IBM_OK unless FAILED) */
  int64_t steps_done; /* steps enqueued for the case */
  double t;           /* simulated time reached */
  double forces[4];   /* as ibm_forces, at the end of the last step */
  double submit_s;    /* host times in seconds since ibm_server_create: */
  double start_s;     /*   admission (case created and classified) */
  double finish_s;    /*   retirement (result read back) */
} ibm_result;

/* device_bytes_budget = 0: 80 % of the device memory free at creation.
 * max_active >= 1, steps_per_chunk >= 1. */
ibm_status ibm_server_create(size_t device_bytes_budget, int max_active, int steps_per_chunk, ibm_server **out);

/* mode: IBM_SERVE_BATCHED | IBM_SERVE_AUTOTUNE (the default), either, or 0
 * (every case on its own stream).  Only before the first submit
 * (IBM_ESTATE afterwards). */
ibm_status ibm_server_set_mode(ibm_server *s, int mode);

/* Counters since creation, n <= IBM_SERVER_NSTATS: [0] group graphs captured,
 * [1] group steps launched, [2] kernels in those steps, [3] autotuner runs,
 * [4] host microseconds spent capturing group graphs and autotuning. */
ibm_status ibm_server_stats(const ibm_server *s, int64_t *out, int n);

/* Queue a request; the arguments are validated and copied (the vertices too).
 * IBM_ENOMEM if the case alone exceeds the budget.  *id receives a positive
 * request id. */
ibm_status ibm_server_submit(ibm_server *s, const ibm_geometry *geometry, const ibm_grid *grid, const ibm_flow *flow,
                             const ibm_motion *motion, int nsteps, int64_t *id);

/* One non-blocking pass of the loop; *n_active / *n_pending (either may be
 * NULL) receive the running and waiting request counts after the pass. */
ibm_status ibm_server_progress(ibm_server *s, int *n_active, int *n_pending);

/* Copy the current record of a request. */
ibm_status ibm_server_poll(ibm_server *s, int64_t id, ibm_result *out);

/* Wait for the running cases, retire them as failed (IBM_ESTATE) and free
 * every resource of the server.  NULL is a no-op. */
ibm_status ibm_server_destroy(ibm_server *s);

#ifdef __cplusplus
}
#endif
#endif
