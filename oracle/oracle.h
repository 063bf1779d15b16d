/*
 * FP64 CPU oracle for the sharp-interface immersed-boundary compressible solver
 * of Seshadri & De, "A Novel Sharp Interface Immersed Boundary Framework for
 * Viscous Flow Simulations at Arbitrary Mach Number Involving Complex and
 * Moving Boundaries" (arXiv 1912.11908).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, obviously-correct
 * restatement of what the paper computes, used to check the CUDA library.  It
 * shares no code, header, table or helper with the CUDA path and must never be
 * linked into, imported by, or called from the product path.  Only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark may load it.
 *
 * Readings of the paper where it is silent are stated next to each function in
 * oracle.c.  Every routine computes in IEEE binary64 with basic operations and
 * sqrt only; the file is built with -ffp-contract=off so that the geometry
 * (classification, tagging, closest features, image points, stencils) is
 * reproducible bit for bit by any IEEE implementation that performs the same
 * operations in the same order.
 *
 * Parity status per function (pins live in tests/test_oracle_*.py):
 *   orc_classify_points  pinned: brute force with exact rationals (Sec. 3.2)
 *   tagging / lists      pinned: independent definition on tiny grids (Sec. 3.2, Sec. 5)
 *   pseudo-normals       pinned: regular polygon radial, bisector property (Sec. 4.2)
 *   closest feature      pinned: dense sampling of the polyline (Sec. 4.1, Eq. 1)
 *   weno5                pinned: polynomial exactness, 5th-order convergence (Sec. 2)
 *   ldfss flux           pinned: consistency F(q,q) = Euler flux, Sod exact Riemann solution (Sec. 2)
 *   viscous flux         pinned: shear-wave and entropy-wave decay rates (Sec. 2)
 *   RK3 + residual       pinned: periodic mass/energy conservation, free-stream preservation
 *   IB reconstruction    pinned: linear-field exactness at a flat wall, quiescent body (Sec. 4.4-4.6, Sec. 5)
 *   quadratic IB / ghost pinned: quadratic-profile exactness at a 45-degree wall whose probes and image points
 *                        fall on cell centres, where the linear form is off (Sec. 4.5, Sec. 5)
 *   forces               pinned: zero force in uniform flow / uniform pressure (Sec. 6, Eq. 9)
 *   drag/lift values     parity unpinned (the paper prints none for these workloads)
 *   3-D residual + RK3   pinned: a field constant along one axis reproduces the 2-D oracle bit for bit in each
 *                        of the three coordinate planes (oracle3d.c)
 *   3-D IB / ghost       pinned: linear profiles at axis-aligned and oblique plane walls, quiescent sphere
 *   3-D forces           pinned: linear pressure and velocity fields on a closed box (per-triangle closed form),
 *                        uniform pressure on the sphere (closed surface, Eq. 9)
 *   3-D CFL rule         pinned: closed form on a uniform state
 */
#ifndef IBM_ORACLE_H
#define IBM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* node tags (Sec. 3.2, Fig. 1; Sec. 5, Fig. 6) */
enum { ORC_FLUID = 0, ORC_SOLID = 1, ORC_IB = 2, ORC_G1 = 3, ORC_G2 = 4, ORC_G3 = 5 };
/* domain sides: 0 x-low, 1 x-high, 2 y-low, 3 y-high */
enum { ORC_BC_FREESTREAM = 0, ORC_BC_OUTFLOW = 1, ORC_BC_PERIODIC = 2 };
enum { ORC_MOTION_STATIC = 0, ORC_MOTION_SIN = 1, ORC_MOTION_CONST = 2, ORC_MOTION_COUPLED = 3, ORC_MOTION_PITCH = 4 };
/* IB nodes: rebuilt from their probes every stage (Sec. 4.4-4.6, the fluid-side nodes of Fig. 1 / Fig. 6),   */
/* or advanced by the flux update like fluid nodes, the wall then imposed by the rebuilt ghost layers alone    */
/* (Sec. 5's field extension).  The second holds normal shocks on blunt bodies where the first lets the mass   */
/* the upwind flux carries into a rebuilt node vanish (M >= 2 stagnation).                                     */
enum { ORC_IB_REBUILD = 0, ORC_IB_ADVANCE = 1 };
enum { ORC_SCHEME_WENO5 = 0, ORC_SCHEME_TVD2 = 1 };
/* IB and ghost reconstruction along the local normal: linear through the wall and one probe / image point     */
/* (the compressible form, Sec. 4.6 and Sec. 5), or quadratic through the wall and two probes / image points    */
/* (the incompressible form, Sec. 4.5 and Sec. 5)                                                               */
enum { ORC_INTERP_LINEAR = 0, ORC_INTERP_QUADRATIC = 1 };
enum { ORC_REGION_FACE = 0, ORC_REGION_VERTEX = 1, ORC_REGION_FALLBACK = 2 };
enum { ORC_TIME_RK3 = 0, ORC_TIME_DUAL = 1 };

typedef struct {
  int nx, ny;              /* cells */
  double x0, x1, y0, y1;   /* domain */
  int bc[4];
  double mach, re, gamma, prandtl, cfl;  /* re <= 0: inviscid */
  double uinf[2];          /* free-stream velocity in units of the reference speed */
  double dt_fixed;         /* > 0: use this time step instead of the CFL rule */
  double ref_len;          /* force normalisation length */
  int nv;                  /* body vertices (closed CCW polyline); 0 = no body */
  const double *verts;     /* 2*nv, interleaved x,y; copied */
  int motion;
  double amp[2], freq, vel[2];  /* COUPLED: vel = initial body velocity */
  double mass;                  /* COUPLED: body mass per unit depth (Eq. 10); RK3 only */
  int ib_mode;                  /* ORC_IB_REBUILD or ORC_IB_ADVANCE */
  /* PITCH (Sec. 7.2): rotation about `pivot`, angle of attack alpha(t) = pitch_mean - pitch_amp cos(2 pi freq t) */
  /* (radians, nose up = clockwise); the given vertices are the body at alpha = 0                                 */
  double pivot[2], pitch_mean, pitch_amp;
  int scheme;                   /* ORC_SCHEME_WENO5 or ORC_SCHEME_TVD2 (Sec. 2: either reconstruction) */
  int time_scheme;         /* ORC_TIME_RK3 or ORC_TIME_DUAL */
  int subiters;            /* dual time: pseudo-time sub-iterations per physical step */
  double dt_phys;          /* dual time: physical time step */
  double cfl_tau;          /* dual time: pseudo-time CFL number */
  int ib_interp;           /* ORC_INTERP_LINEAR or ORC_INTERP_QUADRATIC */
} orc_params;

/* One immersed-boundary or ghost node and its reconstruction stencil. */
typedef struct {
  int32_t cell;      /* j*nx + i */
  int32_t feature;   /* segment index (FACE) or vertex index (VERTEX) */
  int32_t region;    /* ORC_REGION_* */
  int32_t i0, j0;    /* lower-left cell of the interpolation square */
  int32_t mask;      /* bit k: corner k valid; k = 0 (i0,j0), 1 (i0+1,j0), 2 (i0,j0+1), 3 (i0+1,j0+1) */
  int32_t nstep;     /* probe push-outs taken */
  int32_t kind;      /* 0 IB, 1..3 ghost layer */
  double nx, ny;     /* local normal (out of the body) */
  double bx, by;     /* boundary point P' */
  double xi_node;    /* signed distance of the node from P' along the normal */
  double xi_probe;   /* signed distance of the probe / image point from P' */
  double w[4];       /* interpolation weights (0 for invalid corners) */
  double curv;       /* signed curvature 1/R of the surface at P' (convex > 0; Eq. 7) */
  /* QUADRATIC: the second probe / image point, one diagonal spacing beyond the first (mask2 = 0: none found, */
  /* or LINEAR)                                                                                                */
  int32_t i0b, j0b, maskb, nstepb;
  double xi_probe2;
  double wb[4];
} orc_stencil;

typedef struct orc_case orc_case;

orc_case *orc_create(const orc_params *p);
void orc_destroy(orc_case *c);
int orc_classify(orc_case *c);                   /* geometry at the current time */
int orc_step(orc_case *c, int nsteps);           /* RK3 or dual-time physical steps; returns #stencil errors */
void orc_get_state(const orc_case *c, double *dst);      /* [4][ny][nx] conserved */
void orc_set_state(orc_case *c, const double *src);      /* [4][ny][nx] conserved */
void orc_set_time(orc_case *c, double t);                /* tests: pose the body at t from the next classification */
void orc_get_tags(const orc_case *c, uint8_t *dst);      /* [ny][nx] */
int orc_list_len(const orc_case *c, int kind);           /* 0 IB, 1..3 G1..G3 */
void orc_get_list(const orc_case *c, int kind, orc_stencil *dst);
void orc_forces(orc_case *c, double out[4]);             /* Cd, Cl, Fx, Fy */
/* Eq. 9 per segment: surface pressure and skin-friction coefficients at the segment midpoints (NaN where no probe). */
void orc_surface(orc_case *c, double *cp, double *cf);
double orc_time(const orc_case *c);
void orc_body(const orc_case *c, double out[6]);         /* displacement x, y; velocity u, v; last force Fx, Fy */
double orc_last_dt(const orc_case *c);
void orc_reconstruct(orc_case *c, double t);             /* IB + ghost fill at time t (one call of the stage step) */
void orc_vertex_normals(const orc_case *c, double *dst); /* 2*nv */
void orc_closest(const orc_case *c, double px, double py, int32_t *feature, int32_t *region,
                 double *cx, double *cy, double *d2);

/* pure kernels exposed for pins; flux states are (rho, u, v, p) */
void orc_classify_points(int nv, const double *verts, int np, const double *pts, uint8_t *solid);
/* 3-D: closed triangulated surface (verts 3*nv, outward-oriented triangles 3*ntri), points 3*np */
void orc_classify_points_3d(int nv, const double *verts, int ntri, const int *tris, int np, const double *pts,
                            uint8_t *solid);
/* 3-D node tags (ORC_FLUID .. ORC_G3) of an nx*ny*nz lattice, x fastest, from its solid flags */
void orc_tags_3d(int nx, int ny, int nz, const uint8_t *solid, uint8_t *tags);
/* 3-D closest point cp (3*np), pseudo-normal nrm (3*np) and feature kind (0 face, 1 edge, 2 vertex) */
void orc_closest_3d(int nv, const double *verts, int ntri, const int *tris, int np, const double *pts, double *cp,
                    double *nrm, int32_t *kind);
double orc_weno5(const double f[5]);
double orc_tvd2(const double f[3]);
void orc_ldfss_xflux(const double qL[4], const double qR[4], double gamma, double R,
                     double mr2_fixed, double flux[4]);
void orc_euler_xflux(const double q[4], double gamma, double R, double flux[4]);
/* dual time: preconditioning matrix Gamma (Ur) and dW/dQ at Q = (p, u, v, T), row-major 4x4 */
void orc_precond_matrix(const double Q[4], double gamma, double R, double Ur, double out[16]);
void orc_dwdq(const double Q[4], double gamma, double R, double out[16]);
int orc_solve4(const double A[16], const double b[4], double x[4]);

/* ------------------------------------------------------------------------------------------------------ */
/* 3-D flow (oracle3d.c): one uniform block of nx * ny * nz cells with a static closed triangulated body,     */
/* explicit SSP-RK3, the compressible (linear) IB / ghost form.  State (rho, rho u, rho v, rho w, rho E).     */
/* domain sides in bc order: x-low, x-high, y-low, y-high, z-low, z-high                                      */
/* ------------------------------------------------------------------------------------------------------ */
typedef struct {
  int nx, ny, nz;          /* cells */
  double lo[3], hi[3];     /* domain */
  int bc[6];
  double mach, re, gamma, prandtl, cfl;  /* re <= 0: inviscid */
  double uinf[3];
  double dt_fixed;         /* > 0: use this time step instead of the CFL rule */
  double ref_area;         /* force normalisation area */
  int nv, ntri;            /* body: 0 = none */
  const double *verts;     /* 3*nv; copied */
  const int *tris;         /* 3*ntri, counter-clockwise seen from outside; copied */
} orc3_params;

/* One IB or ghost node of the 3-D lattice and its reconstruction stencil. */
typedef struct {
  int32_t node;      /* (k ny + j) nx + i */
  int32_t kind;      /* 0 IB, 1..3 ghost layer */
  int32_t region;    /* closest feature: 0 face, 1 edge, 2 vertex */
  int32_t nstep;     /* probe push-outs taken */
  int32_t i0, j0, k0;/* lowest corner of the interpolation cube */
  int32_t mask;      /* bit b: corner (i0 + (b & 1), j0 + (b >> 1 & 1), k0 + (b >> 2)) valid */
  double n[3];       /* local normal (pseudo-normal of the closest feature, out of the body) */
  double b[3];       /* boundary point P' */
  double xi_node;    /* signed distance of the node from P' along n */
  double xi_probe;   /* signed distance of the probe / image point from P' */
  double w[8];       /* interpolation weights (0 for invalid corners) */
} orc3_stencil;

typedef struct orc3_case orc3_case;

orc3_case *orc3_create(const orc3_params *p);
void orc3_destroy(orc3_case *c);
int orc3_classify(orc3_case *c);                    /* returns #stencil errors */
int orc3_step(orc3_case *c, int nsteps);            /* SSP-RK3 steps; returns #stencil errors */
void orc3_reconstruct(orc3_case *c);                /* IB + ghost fill of the current state (one stage's) */
void orc3_get_state(const orc3_case *c, double *dst);    /* [5][nz][ny][nx] */
void orc3_set_state(orc3_case *c, const double *src);    /* [5][nz][ny][nx] */
void orc3_get_tags(const orc3_case *c, uint8_t *dst);    /* [nz][ny][nx] */
int orc3_list_len(const orc3_case *c, int kind);
void orc3_get_list(const orc3_case *c, int kind, orc3_stencil *dst);
void orc3_forces(orc3_case *c, double out[6]);      /* Cx, Cy, Cz, Fx, Fy, Fz */
double orc3_time(const orc3_case *c);
double orc3_last_dt(const orc3_case *c);

#ifdef __cplusplus
}
#endif
#endif
