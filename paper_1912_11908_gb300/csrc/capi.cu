// C ABI (include/ibm.h): case lifetime, device memory, step orchestration.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <type_traits>

#include "ibm_internal.cuh"

using namespace ibm;

struct ibm_case {
  int device = 0;
  cudaStream_t stream = nullptr;
  Consts k{};
  Geom g{};
  int precision = IBM_PREC_FP64;
  // device memory
  double *vref = nullptr, *vx = nullptr, *vy = nullptr, *snx = nullptr, *sny = nullptr, *vnx = nullptr,
         *vny = nullptr, *vk = nullptr;
  float *segb = nullptr;  // segment bounds of the current pose (stencil searches)
  double *surf = nullptr;  // per segment (Cp, Cf) of the last ibm_surface call
  double *rsnx = nullptr, *rsny = nullptr, *rvnx = nullptr, *rvny = nullptr;  // PITCH: reference-pose normals
  double *A = nullptr, *B = nullptr, *C = nullptr;  // FP64 conserved: state, stage arrays (FP64 mode)
  double *Wn = nullptr, *Wm = nullptr;               // dual time: states at time levels n and n-1
  double *G = nullptr;  // FP32-bulk dual time: the step's constant part of the BDF term (in place of W^{n-1})
  double *Q0 = nullptr;                              // FP32-bulk dual time: (p', u, v, T') of the sub-iteration start
  float *M = nullptr, *F1 = nullptr, *F2 = nullptr;  // FP32-bulk: perturbation mirror and stage arrays
  double *stage64 = nullptr;  // FP32-bulk: absolute-variable staging for ibm_get_state (allocated on first use)
  uint8_t *solid = nullptr, *tag = nullptr;
  int *blockcounts = nullptr;
  ibm_stencil *st = nullptr;
  RStencil32 *rst = nullptr;  // FP32-bulk: compact stencils
  RStencilQ *rsq = nullptr;   // FP32-bulk, quadratic reconstruction: their quadratic part
  int *sid = nullptr;         // FP32-bulk: cell -> stencil index (-1 if none)
  uint8_t *tile_body = nullptr;  // FP32-bulk: stage tiles that rebuild IB / ghost nodes
  int *body_tiles = nullptr;
  int body_cap = 0;
  CUtensorMap tmap[3];              // FP32-bulk: tensor maps of M, F1, F2 for the TMA tile staging
  bool have_tmap = false;           // tensor maps built
  bool use_tma = true;              // stage interior tiles with TMA (ibm_use_tma)
  int plain_variant[2] = {-1, -1};  // FP32-bulk: register budget of the plain stage kernel for stage 1 and for
                                    // stages 2-3 (-1: not tuned yet)
  unsigned int *sch_words = nullptr;  // FP32-bulk explicit: schedule of the persistent step kernel (StepSched)
  bool use_persist = false;           // one persistent launch per step (ibm_use_persistent)
  int stage_launch = 2;               // FP32-bulk explicit stages: 0 plain + body kernels on two streams, 1 one
                                      // kernel, 2 one kernel chained by programmatic launch (ibm_stage_launches)
  bool launch_pinned = false;         // stage_launch set by the caller (else the autotuner picks 0 or 2)
  int step_variant = 0;               // register budget of the persistent kernel
  int step_grid = 0;                  // its grid (0: not computed yet)
  bool autotune = true;
  int box_w = 0, box_h = 0;      // cells spanned by the body's bounding box (any pose), for classification
  cudaStream_t sb = nullptr;     // FP32-bulk: stream of the body-tile kernels (forked from / joined to stream)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // FP32-bulk per-step geometry: after the tags, the stencils run on sb and the force of a body under the fluid
  // force on sf, beside the tile lists and dt on the case stream; joined before the stages
  cudaStream_t sf = nullptr;
  cudaEvent_t ev_tags = nullptr, ev_sten = nullptr, ev_force = nullptr;
  StageBatch *one = nullptr;  // FP32-bulk dual time: the one-case block table of its pseudo-stage launches
  bool geo_forked = false;   // stencils in flight on sb since the last classification
  bool force_forked = false; // force in flight on sf
  int cap = 0;
  bool dt_valid = false;      // FP32-bulk static body: dt of the next step is already in DevState
  DevState *ds = nullptr;
  DevState *hds = nullptr;  // host mirror for read-backs
  char *arena = nullptr;    // every device buffer above except stage64, carved from one stream-ordered allocation
  size_t arena_bytes = 0;
  bool classified = false;
  bool own_stream = false;
  long long launches = 0;
  // CUDA graph of one step (captured on first use)
  bool use_graphs = true;
  cudaGraphExec_t graph = nullptr;
  long long graph_launches = 0;  // kernels per replayed step
  // profiling: event pairs per kernel group
  static constexpr int NGROUP = 6, NEV = 4096;
  bool profiling = false;
  cudaEvent_t ev[NEV] = {};
  int nev = 0;
  int ev_group[NEV / 2] = {};
  bool ev_overflow = false;
};

// record a group boundary (start when begin, end otherwise) while profiling
static void prof_mark(ibm_case *c, int group, bool begin) {
  if (!c->profiling) return;
  if (begin) {
    if (c->nev + 2 > ibm_case::NEV) {
      c->ev_overflow = true;
      return;
    }
    c->ev_group[c->nev / 2] = group;
    cudaEventRecord(c->ev[c->nev], c->stream);
    c->nev++;
  } else {
    if (c->nev % 2 == 0) return;  // start was dropped
    cudaEventRecord(c->ev[c->nev], c->stream);
    c->nev++;
  }
}

static thread_local char g_err[512] = "";

static ibm_status fail(ibm_status s, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return s;
}

#define CU(call)                                                                             \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) return fail(IBM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// Upper bound of IB + ghost nodes: every listed node lies within one cell
// (IB) or three cells (ghost) of the body's bounding box, whatever the pose.
// Axis-aligned box holding the body in every pose it can take: its vertex box (a translating body's pose only
// shifts it), or for a pitching body the disc its vertices sweep about the pivot.
static void body_extent(const ibm_geometry *geo, const ibm_motion *mo, double &xmin, double &xmax, double &ymin,
                        double &ymax) {
  xmin = xmax = geo->verts[0];
  ymin = ymax = geo->verts[1];
  for (int v = 1; v < geo->nverts; v++) {
    xmin = fmin(xmin, geo->verts[2 * v]);
    xmax = fmax(xmax, geo->verts[2 * v]);
    ymin = fmin(ymin, geo->verts[2 * v + 1]);
    ymax = fmax(ymax, geo->verts[2 * v + 1]);
  }
  if (mo && mo->kind == IBM_MOTION_PITCH) {
    double r2 = 0.0;
    for (int v = 0; v < geo->nverts; v++) {
      const double rx = geo->verts[2 * v] - mo->pivot[0], ry = geo->verts[2 * v + 1] - mo->pivot[1];
      r2 = fmax(r2, rx * rx + ry * ry);
    }
    const double r = sqrt(r2);
    xmin = mo->pivot[0] - r;
    xmax = mo->pivot[0] + r;
    ymin = mo->pivot[1] - r;
    ymax = mo->pivot[1] + r;
  }
}

static int list_capacity(const ibm_geometry *geo, const ibm_grid *gr, const ibm_motion *mo) {
  if (!geo || geo->nverts <= 0) return 0;
  double xmin, xmax, ymin, ymax;
  body_extent(geo, mo, xmin, xmax, ymin, ymax);
  double dx = (gr->hi[0] - gr->lo[0]) / gr->nx, dy = (gr->hi[1] - gr->lo[1]) / gr->ny;
  long long w = (long long)ceil((xmax - xmin) / dx) + 10;
  long long h = (long long)ceil((ymax - ymin) / dy) + 10;
  long long c = w * h;
  long long all = (long long)gr->nx * gr->ny;
  if (c > all) c = all;
  return (int)c;
}

static size_t pitch_of(int nx) { return (size_t)((nx + 2 * NG + 31) / 32 * 32); }

// Upper bound of stage tiles (16x16) whose cells or 3-cell halo can hold IB /
// ghost nodes: tiles meeting the body's bounding box grown by 4 cells, for any
// pose (plus one tile per axis for the offset against the tile grid).
static int body_tile_capacity(const ibm_geometry *geo, const ibm_grid *gr, const ibm_motion *mo, int ntiles) {
  if (!geo || geo->nverts <= 0) return 0;
  double xmin, xmax, ymin, ymax;
  body_extent(geo, mo, xmin, xmax, ymin, ymax);
  double dx = (gr->hi[0] - gr->lo[0]) / gr->nx, dy = (gr->hi[1] - gr->lo[1]) / gr->ny;
  long long w = ((long long)ceil((xmax - xmin) / dx) + 8 + 15) / 16 + 2;
  long long h = ((long long)ceil((ymax - ymin) / dy) + 8 + 15) / 16 + 2;
  long long c = w * h;
  return (int)(c < ntiles ? c : ntiles);
}

static ibm_status validate(const ibm_geometry *geo, const ibm_grid *gr, const ibm_flow *fl, const ibm_motion *mo) {
  if (!geo || !gr || !fl) return fail(IBM_EINVAL, "geometry, grid and flow are required");
  if (geo->dim != 2) return fail(IBM_EINVAL, "only dim == 2 bodies are supported");
  if (geo->nverts != 0 && (geo->nverts < 3 || !geo->verts)) return fail(IBM_EINVAL, "body needs >= 3 vertices");
  if (gr->nx < 8 || gr->ny < 8) return fail(IBM_EINVAL, "grid must have at least 8x8 cells");
  if ((long long)gr->nx * gr->ny > (1LL << 30)) return fail(IBM_EINVAL, "grid too large");
  if (!(gr->hi[0] > gr->lo[0]) || !(gr->hi[1] > gr->lo[1])) return fail(IBM_EINVAL, "empty domain");
  for (int s = 0; s < 4; s++)
    if (gr->bc[s] < IBM_BC_FREESTREAM || gr->bc[s] > IBM_BC_PERIODIC) return fail(IBM_EINVAL, "bad bc[%d]", s);
  if ((gr->bc[0] == IBM_BC_PERIODIC) != (gr->bc[1] == IBM_BC_PERIODIC) ||
      (gr->bc[2] == IBM_BC_PERIODIC) != (gr->bc[3] == IBM_BC_PERIODIC))
    return fail(IBM_EINVAL, "periodic sides must come in pairs");
  if (!(fl->mach > 0) || !(fl->gamma > 1) || !(fl->prandtl > 0) || !(fl->ref_len > 0))
    return fail(IBM_EINVAL, "bad flow parameters");
  if (!(fl->cfl > 0) && !(fl->dt_fixed > 0)) return fail(IBM_EINVAL, "cfl or dt_fixed must be positive");
  if (fl->precision != IBM_PREC_FP64 && fl->precision != IBM_PREC_FP32_BULK)
    return fail(IBM_EINVAL, "bad precision");
  if (mo && (mo->kind < IBM_MOTION_STATIC || mo->kind > IBM_MOTION_PITCH)) return fail(IBM_EINVAL, "bad motion");
  if (mo && mo->kind == IBM_MOTION_PITCH && geo->nverts == 0) return fail(IBM_EINVAL, "a pitching motion needs a body");
  if (mo && mo->kind == IBM_MOTION_COUPLED) {
    if (!(mo->mass > 0)) return fail(IBM_EINVAL, "a body moving under the fluid force needs mass > 0");
    if (fl->time_scheme != IBM_TIME_RK3) return fail(IBM_EINVAL, "a body moving under the fluid force needs RK3");
    if (geo->nverts == 0) return fail(IBM_EINVAL, "a body moving under the fluid force needs a body");
  }
  if (fl->time_scheme != IBM_TIME_RK3 && fl->time_scheme != IBM_TIME_DUAL) return fail(IBM_EINVAL, "bad time scheme");
  if (fl->ib_mode != IBM_IB_REBUILD && fl->ib_mode != IBM_IB_ADVANCE) return fail(IBM_EINVAL, "bad ib_mode");
  if (fl->scheme != IBM_SCHEME_WENO5 && fl->scheme != IBM_SCHEME_TVD2) return fail(IBM_EINVAL, "bad scheme");
  if (fl->ib_interp != IBM_INTERP_LINEAR && fl->ib_interp != IBM_INTERP_QUADRATIC)
    return fail(IBM_EINVAL, "bad ib_interp");
  if (fl->time_scheme == IBM_TIME_DUAL) {
    if (!(fl->dt_phys > 0) || !(fl->cfl_tau > 0) || fl->subiters < 1)
      return fail(IBM_EINVAL, "dual time needs dt_phys > 0, cfl_tau > 0, subiters >= 1");
  }
  return IBM_OK;
}

// Assign every device buffer of the case an offset in one allocation starting
// at base (NULL: only count) and return the total size.  Buffers start on
// 256-byte boundaries.
static size_t carve(ibm_case *c, char *base) {
  const Consts &k = c->k;
  const size_t ncell = (size_t)k.nx * k.ny, plane = (size_t)k.plane;
  const size_t nv = c->g.nv > 0 ? (size_t)c->g.nv : 1;
  size_t off = 0;
  auto take = [&](auto **p, size_t n) {
    using T = typename std::remove_reference<decltype(**p)>::type;
    *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += (n * sizeof(T) + 255) & ~(size_t)255;
  };
  take(&c->vref, 2 * nv);
  take(&c->vx, nv);
  take(&c->vy, nv);
  take(&c->snx, nv);
  take(&c->sny, nv);
  take(&c->vnx, nv);
  take(&c->vny, nv);
  take(&c->vk, nv);
  take(&c->segb, 3 * nv);
  take(&c->surf, 2 * nv);
  if (k.motion.kind == IBM_MOTION_PITCH) {
    take(&c->rsnx, nv);
    take(&c->rsny, nv);
    take(&c->rvnx, nv);
    take(&c->rvny, nv);
  }
  take(&c->A, 4 * plane);
  if (c->precision == IBM_PREC_FP64) {
    take(&c->B, 4 * plane);
    take(&c->C, 4 * plane);
    if (k.dual) {
      take(&c->Wn, 4 * plane);
      take(&c->Wm, 4 * plane);
    }
  } else {
    take(&c->M, 4 * plane);
    take(&c->F1, 4 * plane);
    take(&c->F2, 4 * plane);
    if (k.dual) {  // FP64 pseudo-stage iterates, time level n, BDF part, primitives of the sub-iteration's start
      take(&c->B, 4 * plane);
      take(&c->C, 4 * plane);
      take(&c->Wn, 4 * plane);
      take(&c->G, 4 * plane);
      take(&c->Q0, 4 * plane);
    }
    take(&c->rst, (size_t)(c->cap > 0 ? c->cap : 1));
    if (k.quad) take(&c->rsq, (size_t)(c->cap > 0 ? c->cap : 1));
    take(&c->sid, ncell);
    take(&c->tile_body, (size_t)stage_tiles(k));
    take(&c->body_tiles, (size_t)(c->body_cap > 0 ? c->body_cap : 1));
    if (!k.dual) take(&c->sch_words, step_sched_bytes(k) / sizeof(unsigned int));
  }
  take(&c->solid, ncell);
  take(&c->tag, ncell);
  take(&c->blockcounts, 4 * ((ncell + 1023) / 1024));
  take(&c->st, (size_t)(c->cap > 0 ? c->cap : 1));
  take(&c->ds, 1);
  return off;
}

// Host-side set-up of a case from validated arguments: constants, list and
// tile capacities, the body's bounding-box extent in cells.
static void init_case(ibm_case *c, const ibm_geometry *geo, const ibm_grid *gr, const ibm_flow *fl,
                      const ibm_motion *mo) {
  c->precision = fl->precision;
  Consts &k = c->k;
  k.nx = gr->nx;
  k.ny = gr->ny;
  k.pitch = (int)pitch_of(gr->nx);
  k.rows = gr->ny + 2 * NG;
  k.plane = (long long)k.pitch * k.rows;
  k.x0 = gr->lo[0];
  k.y0 = gr->lo[1];
  k.dx = (gr->hi[0] - gr->lo[0]) / gr->nx;
  k.dy = (gr->hi[1] - gr->lo[1]) / gr->ny;
  k.h = sqrt(k.dx * k.dx + k.dy * k.dy);
  k.dmin = k.dx < k.dy ? k.dx : k.dy;
  k.gamma = fl->gamma;
  k.pinf = 1.0 / (fl->gamma * fl->mach * fl->mach);
  k.R = k.pinf;
  k.cp = k.gamma * k.R / (k.gamma - 1.0);
  k.iR = 1.0 / k.R;
  k.ig1 = 1.0 / (k.gamma - 1.0);
  k.mu = fl->re > 0.0 ? 1.0 / fl->re : 0.0;
  k.kappa = k.mu * k.cp / fl->prandtl;
  k.prandtl = fl->prandtl;
  k.cfl = fl->cfl;
  k.dt_fixed = fl->dt_fixed;
  k.ref_len = fl->ref_len;
  k.uinf[0] = fl->uinf[0];
  k.uinf[1] = fl->uinf[1];
  k.Uinf[0] = 1.0;
  k.Uinf[1] = fl->uinf[0];
  k.Uinf[2] = fl->uinf[1];
  k.Uinf[3] = k.pinf / (k.gamma - 1.0) + 0.5 * (fl->uinf[0] * fl->uinf[0] + fl->uinf[1] * fl->uinf[1]);
  k.Hinf = k.gamma / (k.gamma - 1.0) * k.pinf + 0.5 * (fl->uinf[0] * fl->uinf[0] + fl->uinf[1] * fl->uinf[1]);
  for (int s = 0; s < 4; s++) k.bc[s] = gr->bc[s];
  k.motion.kind = mo ? mo->kind : IBM_MOTION_STATIC;
  for (int d = 0; d < 2; d++) {
    k.motion.amp[d] = mo ? mo->amp[d] : 0.0;
    k.motion.vel[d] = mo ? mo->vel[d] : 0.0;
  }
  k.motion.freq = mo ? mo->freq : 0.0;
  k.motion.mass = mo && mo->kind == IBM_MOTION_COUPLED ? mo->mass : 0.0;
  for (int d = 0; d < 2; d++) k.motion.pivot[d] = mo && mo->kind == IBM_MOTION_PITCH ? mo->pivot[d] : 0.0;
  k.motion.pmean = mo && mo->kind == IBM_MOTION_PITCH ? mo->pitch_mean : 0.0;
  k.motion.pamp = mo && mo->kind == IBM_MOTION_PITCH ? mo->pitch_amp : 0.0;
  k.dual = fl->time_scheme == IBM_TIME_DUAL;
  k.ib_advance = fl->ib_mode == IBM_IB_ADVANCE;
  k.tvd2 = fl->scheme == IBM_SCHEME_TVD2;
  k.quad = fl->ib_interp == IBM_INTERP_QUADRATIC;
  k.subiters = fl->subiters;
  k.dt_phys = fl->dt_phys;
  k.idt_phys = fl->dt_phys > 0.0 ? 1.0 / fl->dt_phys : 0.0;
  k.cfl_tau = fl->cfl_tau;
  c->g.nv = geo->nverts;
  c->cap = list_capacity(geo, gr, mo);
  if (c->precision == IBM_PREC_FP32_BULK) c->body_cap = body_tile_capacity(geo, gr, mo, stage_tiles(k));
  if (geo->nverts > 0) {
    double xmin, xmax, ymin, ymax;
    body_extent(geo, mo, xmin, xmax, ymin, ymax);
    c->box_w = (int)fmin((double)k.nx, ceil((xmax - xmin) / k.dx) + 4);
    c->box_h = (int)fmin((double)k.ny, ceil((ymax - ymin) / k.dy) + 4);
  }
}

extern "C" size_t ibm_case_device_bytes(const ibm_geometry *geo, const ibm_grid *gr, const ibm_flow *fl,
                                        const ibm_motion *mo) {
  if (validate(geo, gr, fl, mo) != IBM_OK) return 0;
  ibm_case *c = new (std::nothrow) ibm_case();
  if (!c) {
    fail(IBM_ENOMEM, "host allocation failed");
    return 0;
  }
  init_case(c, geo, gr, fl, mo);
  size_t b = carve(c, nullptr);
  delete c;
  return b;
}

// Stream-ordered release: nothing here waits for the device, so cases can be
// retired while other cases run.
static void free_case(ibm_case *c) {
  if (!c) return;
  delete c->one;
  if (c->stage64) cudaFreeAsync(c->stage64, c->stream);
  if (c->arena) cudaFreeAsync(c->arena, c->stream);
  delete c->hds;
  if (c->graph) cudaGraphExecDestroy(c->graph);
  for (int q = 0; q < ibm_case::NEV; q++)
    if (c->ev[q]) cudaEventDestroy(c->ev[q]);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  for (cudaEvent_t ev : {c->ev_tags, c->ev_sten, c->ev_force})
    if (ev) cudaEventDestroy(ev);
  if (c->sb) cudaStreamDestroy(c->sb);
  if (c->sf) cudaStreamDestroy(c->sf);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

__global__ void k_fill(double *p, size_t n, double v0, double v1, double v2, double v3) {
  const size_t q = n / 4;
  for (size_t m = blockIdx.x * (size_t)blockDim.x + threadIdx.x; m < n; m += (size_t)gridDim.x * blockDim.x) {
    const size_t v = m / q;
    p[m] = v == 0 ? v0 : v == 1 ? v1 : v == 2 ? v2 : v3;
  }
}

// the four planes of p set to the four values (n = 4 planes)
static cudaError_t fill4(double *p, size_t n, const double *v, cudaStream_t s) {
  k_fill<<<4 * 152, 256, 0, s>>>(p, n, v[0], v[1], v[2], v[3]);
  return cudaGetLastError();
}

extern "C" ibm_status ibm_create_case(const ibm_geometry *geo, const ibm_grid *gr, const ibm_flow *fl,
                                      const ibm_motion *mo, void *stream, ibm_case **out) {
  if (!out) return fail(IBM_EINVAL, "out is NULL");
  *out = nullptr;
  ibm_status st = validate(geo, gr, fl, mo);
  if (st != IBM_OK) return st;
  ibm_case *c = new (std::nothrow) ibm_case();
  if (!c) return fail(IBM_ENOMEM, "host allocation failed");
  cudaGetDevice(&c->device);
  prepare_geometry_kernels();
  c->stream = (cudaStream_t)stream;
  if (!c->stream) {
    if (cudaStreamCreate(&c->stream) != cudaSuccess) {
      delete c;
      cudaGetLastError();
      return fail(IBM_ECUDA, "stream creation failed");
    }
    c->own_stream = true;
  }
  init_case(c, geo, gr, fl, mo);
  const Consts &k = c->k;
  const int nv = geo->nverts;
  const size_t ncell = (size_t)k.nx * k.ny;
  const size_t plane = (size_t)k.plane;
  cudaStream_t s = c->stream;

  c->arena_bytes = carve(c, nullptr);
  cudaError_t e = cudaMallocAsync((void **)&c->arena, c->arena_bytes, s);
  if (e == cudaSuccess) carve(c, c->arena);
  else c->arena = nullptr;
  c->hds = new (std::nothrow) DevState();
  if (e == cudaSuccess && !c->hds) e = cudaErrorMemoryAllocation;
  if (e == cudaSuccess && c->precision == IBM_PREC_FP32_BULK) {
    // body tiles are on the critical path of every stage: give their stream the highest priority
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    e = cudaStreamCreateWithPriority(&c->sb, cudaStreamNonBlocking, prio_hi);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&c->sf, cudaStreamNonBlocking, prio_hi);
    for (cudaEvent_t *ev : {&c->ev_tags, &c->ev_sten, &c->ev_force})
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    free_case(c);
    cudaGetLastError();
    return fail(IBM_ENOMEM, "device allocation failed: %s", cudaGetErrorString(e));
  }
  c->g.vref = c->vref;
  c->g.vx = c->vx;
  c->g.vy = c->vy;
  c->g.snx = c->snx;
  c->g.sny = c->sny;
  c->g.vnx = c->vnx;
  c->g.vny = c->vny;
  c->g.vk = c->vk;
  c->g.sb = c->segb;
  c->g.rsq = c->rsq;
  {  // stencil searches: half a warp per node when the body's nodes (about four layers along its perimeter)
     // fill the GPU with whole-warp nodes, a whole warp otherwise
    double perim = 0.0;
    for (int v = 0; v < c->g.nv; v++) {
      const int v1 = v + 1 == c->g.nv ? 0 : v + 1;
      perim += std::hypot(geo->verts[2 * v1] - geo->verts[2 * v], geo->verts[2 * v1 + 1] - geo->verts[2 * v + 1]);
    }
    const double cells = perim / std::min(k.dx, k.dy);
    c->g.stencil_lanes = 4.0 * cells >= 4.0 * 2 * 152 ? 16 : 32;
  }
  const bool pitching = k.motion.kind == IBM_MOTION_PITCH;
  c->g.rsnx = pitching ? c->rsnx : nullptr;
  c->g.rsny = pitching ? c->rsny : nullptr;
  c->g.rvnx = pitching ? c->rvnx : nullptr;
  c->g.rvny = pitching ? c->rvny : nullptr;

  ibm_status rs = IBM_OK;
  do {
    if (nv > 0) {
      if (cudaMemcpyAsync(c->vref, geo->verts, sizeof(double) * 2 * nv, cudaMemcpyHostToDevice, s) != cudaSuccess) {
        rs = fail(IBM_ECUDA, "vertex upload failed");
        break;
      }
      // normals of the reference pose: the current pose's for a translating body; a pitching body's pose
      // kernel rotates them into the current arrays at every classification
      if (pitching)
        launch_normals(nv, c->vref, c->rsnx, c->rsny, c->rvnx, c->rvny, c->vk, s);
      else
        launch_normals(nv, c->vref, c->snx, c->sny, c->vnx, c->vny, c->vk, s);
      c->launches++;
    }
    std::memset(c->hds, 0, sizeof(DevState));
    if (k.motion.kind == IBM_MOTION_COUPLED)
      for (int d = 0; d < 2; d++) c->hds->bV[d] = k.motion.vel[d];  // at rest where it starts, moving at vel
    if (k.dt_fixed > 0.0 || k.dual) {
      c->hds->dt = k.dual ? k.dt_phys : k.dt_fixed;
      c->hds->dtf = (float)c->hds->dt;
    }
    // (the copy from pageable memory is staged before the call returns)
    // fluid, untagged and unlisted everywhere (the geometry kernels keep that outside the body's rectangle)
    if (cudaMemcpyAsync(c->ds, c->hds, sizeof(DevState), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(c->tag, 0, ncell, s) != cudaSuccess || cudaMemsetAsync(c->solid, 0, ncell, s) != cudaSuccess ||
        (c->sid && cudaMemsetAsync(c->sid, 0xff, ncell * sizeof(int), s) != cudaSuccess) ||
        (c->sch_words && cudaMemsetAsync(c->sch_words, 0, step_sched_bytes(k), s) != cudaSuccess)) {
      rs = fail(IBM_ECUDA, "state initialisation failed");
      break;
    }
    // free stream everywhere (halo included); the FP32-bulk FP64 state holds dU = U - U_inf
    const double zero[4] = {0.0, 0.0, 0.0, 0.0};
    const double *u0 = c->precision == IBM_PREC_FP32_BULK ? zero : k.Uinf;
    for (double *w : {c->A, c->B, c->C, c->Wn, c->Wm})
      if (w && fill4(w, 4 * plane, u0, s) != cudaSuccess) rs = fail(IBM_ECUDA, "state initialisation failed");
    if (rs != IBM_OK) break;
    if (c->M) {
      for (float *p : {c->M, c->F1, c->F2})
        if (cudaMemsetAsync(p, 0, 4 * plane * sizeof(float), s) != cudaSuccess) rs = fail(IBM_ECUDA, "memset failed");
    }
    for (double *w : {c->A, c->B, c->C, c->Wn, c->Wm})
      if (w) c->launches += 1;
    if (c->precision == IBM_PREC_FP32_BULK) {
      float *const arrays[3] = {c->M, c->F1, c->F2};
      c->have_tmap = make_stage_tmaps(k, arrays, c->tmap);
    }

  } while (0);
  if (rs != IBM_OK) {
    free_case(c);
    return rs;
  }
  *out = c;
  return IBM_OK;
}

// the per-step geometry work forked by do_classify (stencils) and enqueue_force (force) joins the case stream
static void geometry_join(ibm_case *c) {
  if (c->geo_forked) {
    cudaEventRecord(c->ev_sten, c->sb);
    cudaStreamWaitEvent(c->stream, c->ev_sten, 0);
    c->geo_forked = false;
  }
  if (c->force_forked) {
    cudaEventRecord(c->ev_force, c->sf);
    cudaStreamWaitEvent(c->stream, c->ev_force, 0);
    c->force_forked = false;
  }
}

// Eq. 9-10: the force at the start of the step sets the body's acceleration; beside the stencils when the
// classification forked them (both read only the tags, the state and the pose)
static int enqueue_force(ibm_case *c) {
  const bool f64 = c->precision == IBM_PREC_FP64;
  if (c->geo_forked) {
    cudaStreamWaitEvent(c->sf, c->ev_tags, 0);
    launch_forces_f64(c->k, c->g, c->tag, c->A, !f64, c->ds, c->sf, true);
    c->force_forked = true;
  } else {
    launch_forces_f64(c->k, c->g, c->tag, c->A, !f64, c->ds, c->stream, true);
  }
  return 1;
}

// Classification of the current pose.  defer_join: a case with a side stream
// leaves its stencils running there (geo_forked) for the caller to overlap
// with other pre-stage work and join (geometry_join) before the stages.
static ibm_status do_classify(ibm_case *c, bool defer_join = false) {
  cudaStream_t s = c->stream;
  int nl = 0;
  prof_mark(c, 4, true);
  if (c->g.nv > 0 && c->g.nv <= FUSED_MAX_VERTS) {
    // pose + classification, tags / lists / tile lists, stencils: three kernels over the body's rectangle
    nl += launch_fused_geometry(c->k, c->g, c->solid, c->tag, c->st, c->cap, c->rst, c->sid, c->tile_body,
                                c->body_tiles, c->body_cap, c->box_w, c->box_h, c->ds, c->blockcounts, s, c->sb,
                                c->ev_tags);
    c->geo_forked = c->sb != nullptr && c->cap > 0;
    if (!defer_join) {
      geometry_join(c);
      prof_mark(c, 4, false);
    }
    c->launches += nl;
    c->classified = true;
    CU(cudaGetLastError());
    return IBM_OK;
  }
  if (c->g.nv > 0) {
    launch_pose(c->k, c->g, c->ds, s);
    launch_classify(c->k, c->g, c->solid, c->ds, c->box_w, c->box_h, s);
    nl += 2;
  } else {
    cudaMemsetAsync(c->solid, 0, (size_t)c->k.nx * c->k.ny, s);
    if (c->sid) cudaMemsetAsync(c->sid, 0xff, sizeof(int) * (size_t)c->k.nx * c->k.ny, s);
  }
  launch_tags(c->k, c->solid, c->tag, c->blockcounts, c->ds, c->cap, c->st, s, &nl);
  if (c->g.nv > 0) {
    launch_stencils(c->k, c->g, c->tag, c->st, c->cap, c->ds, s);
    nl += 1;
    if (c->rst) {
      launch_compact_stencils(c->k, c->st, c->rst, c->rsq, c->sid, c->cap, c->ds, s);
      nl += 1;
    }
  }
  if (c->tile_body) {
    launch_tile_lists(c->k, c->tag, c->tile_body, c->body_tiles, c->body_cap, c->ds, c->g.nv > 0, s);
    nl += 2;
  }
  if (!defer_join) prof_mark(c, 4, false);
  c->launches += nl;
  c->classified = true;
  CU(cudaGetLastError());
  return IBM_OK;
}

extern "C" ibm_status ibm_classify(ibm_case *c) {
  if (!c) return fail(IBM_EINVAL, "case is NULL");
  return do_classify(c);
}

// FP32-bulk with a static body and the CFL rule: the last stage of each step
// computes the next step's dt (the fluid set cannot change between steps)
static bool fused_cfl(const ibm_case *c) {
  return c->precision == IBM_PREC_FP32_BULK && c->k.motion.kind == IBM_MOTION_STATIC && !(c->k.dt_fixed > 0.0) &&
         !c->k.dual;
}

// the explicit FP32-bulk step runs as one persistent launch
static bool persistent_step(const ibm_case *c) {
  return c->use_persist && c->sch_words && c->precision == IBM_PREC_FP32_BULK && !c->k.dual && !c->k.tvd2 &&
         !c->k.quad;
}

// one explicit step on the case stream (kernels only; graph-capturable)
static int enqueue_step(ibm_case *c) {
  cudaStream_t s = c->stream;
  int nl = 0;
  // with a side stream the classification's stencils (and the force of a body under the fluid force) overlap
  // the other pre-stage work; the profile's geometry group then spans all of it, up to the join
  bool geo_open = false;
  if (!c->classified || c->k.motion.kind != IBM_MOTION_STATIC) {
    int before = (int)c->launches;
    geo_open = c->sb != nullptr;
    do_classify(c, geo_open);
    nl += (int)c->launches - before;
    c->launches = before;
  }
  auto join = [&]() {
    geometry_join(c);
    if (geo_open) prof_mark(c, 4, false);
    geo_open = false;
  };
  if (c->k.dual) {
    // dual time: W^{n-1} <- W^n <- W, then sub-iterations of three pseudo stages at t + dt
    double *din[3] = {c->A, c->B, c->C};
    double *dout[3] = {c->B, c->C, c->A};
    if (c->precision == IBM_PREC_FP32_BULK) {
      // the time levels enter the pseudo stages only through the BDF part G, formed once per physical step
      launch_dual_levels(c->k, c->A, c->Wn, c->G, c->ds, s);
      nl += 1;
      join();
      // FP32 residual of the mirror, FP64 point-implicit update; IB / ghost nodes rebuilt in the tile loads
      float *fin[3] = {c->M, c->F1, c->F2};
      float *fout[3] = {c->F1, c->F2, c->M};
      // one launch per pseudo stage: the block-table kernel of the request loop with this case alone in the
      // table (so that a case gives the same bits alone and in a group); TVD-2 and the quadratic reconstruction
      // their own kernels.  The table (kernel parameters; its pointers fixed for the case's life) is built once.
      const StageBatch *one = nullptr;
      if (c->stage_launch > 0 && !c->k.tvd2 && !c->k.quad) {
        if (!c->one) {
          StageCase sc;
          case_stage_desc(c, &sc);
          c->one = new (std::nothrow) StageBatch();
          if (c->one) build_stage_batch(&sc, 1, c->one);
        }
        one = c->one;
      }
      for (int it = 0; it < c->k.subiters; it++)
        for (int st = 1; st <= 3; st++) {
          prof_mark(c, 0, true);
          // one launch per pseudo stage (form 2: chained by programmatic launch); the two-stream form otherwise,
          // and if the table could not be allocated
          if (c->stage_launch > 0 && (one || c->k.tvd2 || c->k.quad)) {
            if (one)
              launch_dual_f32_batch_one(*one, st, 0, c->stage_launch == 2, s);
            else
              launch_dual_f32_var(c->k, st, fin[st - 1], fout[st - 1], c->A, din[st - 1], dout[st - 1], c->G,
                                  c->Q0, c->tag, c->sid, c->rst, c->tile_body, c->body_tiles, c->body_cap, c->ds,
                                  c->stage_launch == 2, s, c->rsq);
            nl += 1;
          } else {
            cudaEventRecord(c->ev_fork, s);
            cudaStreamWaitEvent(c->sb, c->ev_fork, 0);
            launch_dual_f32(c->k, st, fin[st - 1], fout[st - 1], c->A, din[st - 1], dout[st - 1], c->G, c->Q0,
                            c->tag, c->sid, c->rst, c->tile_body, c->body_tiles, c->body_cap, c->ds, s, c->sb,
                            c->rsq);
            cudaEventRecord(c->ev_join, c->sb);
            cudaStreamWaitEvent(s, c->ev_join, 0);
            nl += 1 + (c->body_cap > 0);
          }
          prof_mark(c, 0, false);
        }
      launch_dual_end(c->k, c->ds, s);
      return nl + 1;
    }
    join();
    const size_t bytes = 4 * (size_t)c->k.plane * sizeof(double);
    cudaMemcpyAsync(c->Wm, c->Wn, bytes, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(c->Wn, c->A, bytes, cudaMemcpyDeviceToDevice, s);
    for (int it = 0; it < c->k.subiters; it++)
      for (int st = 1; st <= 3; st++) {
        prof_mark(c, 1, true);
        launch_recon_f64(c->k, din[st - 1], c->st, c->cap, c->ds, 2, s, &nl);
        prof_mark(c, 1, false);
        prof_mark(c, 0, true);
        launch_dual_f64(c->k, st, c->A, din[st - 1], dout[st - 1], c->Wn, c->Wm, c->tag, c->ds, s);
        prof_mark(c, 0, false);
        nl += 1;
      }
    launch_dual_end(c->k, c->ds, s);
    return nl + 1;
  }
  const bool f64 = c->precision == IBM_PREC_FP64;
  const bool fuse_cfl = fused_cfl(c);
  const bool coupled = c->k.motion.kind == IBM_MOTION_COUPLED;
  if (coupled) {  // Eq. 10: the force at the start of the step sets the body's acceleration for the step
    if (!geo_open) prof_mark(c, 4, true);
    nl += enqueue_force(c);
    if (!geo_open) prof_mark(c, 4, false);
  }
  if (!geo_open) prof_mark(c, 3, true);
  if (f64) launch_dt(c->k, c->A, c->tag, c->ds, s, &nl);
  else if (!fuse_cfl) launch_dt_f32(c->k, c->M, c->tag, c->ds, s, &nl);
  if (!geo_open) prof_mark(c, 3, false);
  join();
  if (!f64 && persistent_step(c)) {
    // the three stages in one launch (the end of the step and the next dt included)
    if (!c->step_grid) c->step_grid = step_f32_grid(c->k, c->step_variant);
    prof_mark(c, 0, true);
    launch_step_f32(c->k, c->M, c->F1, c->F2, c->A, c->tag, c->sid, c->rst, c->tile_body, c->body_tiles,
                    c->body_cap, c->ds, reinterpret_cast<StepSched *>(c->sch_words), fuse_cfl,
                    c->have_tmap && c->use_tma ? c->tmap : nullptr, c->step_variant, c->step_grid, 1, 3, s);
    prof_mark(c, 0, false);
    if (coupled) {
      launch_body_end(c->ds, s);
      nl += 1;
    }
    return nl + 1;
  }
  double *in64[3] = {c->A, c->B, c->C};
  double *out64[3] = {c->B, c->C, c->A};
  float *in32[3] = {c->M, c->F1, c->F2};
  float *out32[3] = {c->F1, c->F2, nullptr};
  for (int st = 1; st <= 3; st++) {
    if (f64) {
      prof_mark(c, 1, true);
      launch_recon_f64(c->k, in64[st - 1], c->st, c->cap, c->ds, st, s, &nl);
      prof_mark(c, 1, false);
    }
    // domain halos (and, in FP32-bulk mode, IB / ghost nodes) are applied
    // inside the stage kernel's tile load; the end of the step (t += dt) is
    // folded into stage 3
    prof_mark(c, 0, true);
    const int pv = c->plain_variant[st == 1 ? 0 : 1] < 0 ? 0 : c->plain_variant[st == 1 ? 0 : 1];
    if (f64) launch_stage_f64(c->k, st, c->A, in64[st - 1], out64[st - 1], c->tag, c->ds, s);
    else if (c->stage_launch > 0) {
      // one launch for all tiles of the stage (body-tile slots first)
      launch_stage_f32_one(c->k, st, c->M, in32[st - 1], out32[st - 1], c->A, c->tag, c->sid, c->rst, c->tile_body,
                           c->body_tiles, c->body_cap, c->ds, fuse_cfl, pv,
                           c->have_tmap && c->use_tma ? &c->tmap[st - 1] : nullptr, c->stage_launch == 2, s,
                           c->rsq);
    } else {
      // body tiles run on a forked stream, concurrently with the plain tiles
      cudaEventRecord(c->ev_fork, s);
      cudaStreamWaitEvent(c->sb, c->ev_fork, 0);
      launch_stage_f32(c->k, st, c->M, in32[st - 1], out32[st - 1], c->A, c->tag, c->sid, c->rst, c->tile_body,
                       c->body_tiles, c->body_cap, c->ds, fuse_cfl, s, c->sb, pv, true,
                       c->have_tmap && c->use_tma ? &c->tmap[st - 1] : nullptr, c->rsq);
      cudaEventRecord(c->ev_join, c->sb);
      cudaStreamWaitEvent(s, c->ev_join, 0);
      if (c->body_cap > 0) nl += 1;
    }
    prof_mark(c, 0, false);
    nl += 1;
  }
  if (coupled) {  // Eq. 10: position and velocity over the step (t has advanced in stage 3)
    prof_mark(c, 5, true);
    launch_body_end(c->ds, s);
    prof_mark(c, 5, false);
    nl += 1;
  }
  return nl;
}

// Autotuner of the FP32-bulk step: for each launch form (plain-tile and
// body-tile kernels on two streams; one kernel per stage with programmatic
// launch) and each register budget, time repeated launches of stage 1 and of
// stage 2 as the step runs them, in interleaved rounds keeping each
// candidate's best time; per form the best budget per stage group, then the
// form with the shorter step (stage 3 takes stage 2's choice).  Picked once
// per device, grid size and pinned form for the whole process.  Between steps stages
// 1 and 2 leave the solution unchanged: they read the mirror of U^n (and the
// stage-1 array) and write the stage arrays, the stage times, and U^n on IB /
// ghost nodes with the values the step's own stage 1 writes again.
static std::mutex g_tune_mu;
struct Tuned {
  int v1, v2, launch;
};
static std::map<std::tuple<int, int, int, int>, Tuned> g_tuned;

static ibm_status tune_plain_variant(ibm_case *c) {
  if (c->precision != IBM_PREC_FP32_BULK || c->plain_variant[0] >= 0) return IBM_OK;
  if (!c->autotune || c->k.dual) {  // dual time has its own kernels
    c->plain_variant[0] = c->plain_variant[1] = 0;
    return IBM_OK;
  }
  // candidates: the register budgets of the launch form the caller pinned, or of both forms (two-stream plain and
  // body kernels; one kernel per stage with programmatic launch)
  const auto key = std::make_tuple(c->device, c->k.nx, c->k.ny, c->launch_pinned ? c->stage_launch : -1);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      c->plain_variant[0] = it->second.v1;
      c->plain_variant[1] = it->second.v2;
      c->stage_launch = it->second.launch;
      return IBM_OK;
    }
  }
  int forms[2] = {c->stage_launch, -1}, nforms = 1;
  if (!c->launch_pinned) {
    forms[0] = 2;
    forms[1] = 0;
    nforms = 2;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  const bool fuse = fused_cfl(c);
  cudaStream_t s = c->stream;
  auto pair = [&](int stage, int v, int form) {
    const CUtensorMap *tm = c->have_tmap && c->use_tma ? &c->tmap[stage - 1] : nullptr;
    if (form > 0) {
      launch_stage_f32_one(c->k, stage, c->M, stage == 1 ? c->M : c->F1, stage == 1 ? c->F1 : c->F2, c->A, c->tag,
                           c->sid, c->rst, c->tile_body, c->body_tiles, c->body_cap, c->ds, fuse, v, tm, form == 2, s,
                           c->rsq);
      return;
    }
    cudaEventRecord(c->ev_fork, s);
    cudaStreamWaitEvent(c->sb, c->ev_fork, 0);
    launch_stage_f32(c->k, stage, c->M, stage == 1 ? c->M : c->F1, stage == 1 ? c->F1 : c->F2, c->A, c->tag, c->sid,
                     c->rst, c->tile_body, c->body_tiles, c->body_cap, c->ds, fuse, s, c->sb, v, true, tm, c->rsq);
    cudaEventRecord(c->ev_join, c->sb);
    cudaStreamWaitEvent(s, c->ev_join, 0);
  };
  constexpr int ROUNDS = 5, REPS = 8;
  float best[2][2][PLAIN_VARIANTS];  // form, stage, variant
  for (int f = 0; f < 2; f++)
    for (int st = 0; st < 2; st++)
      for (int v = 0; v < PLAIN_VARIANTS; v++) best[f][st][v] = 1e30f;
  pair(1, 0, forms[0]);  // stage-1 array for the stage-2 timings
  long long nl = 1 + (c->body_cap > 0 && forms[0] == 0);
  cudaError_t e = cudaSuccess;
  for (int round = 0; round < ROUNDS && e == cudaSuccess; round++)
    for (int f = 0; f < nforms && e == cudaSuccess; f++)
      for (int st = 0; st < 2 && e == cudaSuccess; st++)
        for (int v = 0; v < PLAIN_VARIANTS && e == cudaSuccess; v++) {
          pair(st + 1, v, forms[f]);  // warm-up
          cudaEventRecord(e0, s);
          for (int rep = 0; rep < REPS; rep++) pair(st + 1, v, forms[f]);
          cudaEventRecord(e1, s);
          nl += (REPS + 1) * (1 + (c->body_cap > 0 && forms[f] == 0));
          float ms = 0.f;
          e = cudaEventSynchronize(e1);
          if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
          if (e == cudaSuccess && ms < best[f][st][v]) best[f][st][v] = ms;
        }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return fail(IBM_ECUDA, "autotuning failed: %s", cudaGetErrorString(e));
  // per form the best budget per stage group; the form with the shorter step (stage 3 runs stage 2's choice)
  int pick[2][2];
  float step_ms[2];
  for (int f = 0; f < nforms; f++) {
    for (int st = 0; st < 2; st++) {
      // another budget replaces the compiler's default only when it is clearly faster: margins within the
      // timing noise flip between runs (a 2% margin still flipped the stage-1 pick at 768 x 384 on GB300,
      // and the pick that won by that margin made flushed-cache steps 4% slower), and the default keeps more
      // blocks resident for cold caches
      int b = 0;
      for (int v = 1; v < PLAIN_VARIANTS; v++)
        if (best[f][st][v] < (b == 0 ? 0.96f : 1.f) * best[f][st][b]) b = v;
      pick[f][st] = b;
    }
    step_ms[f] = best[f][0][pick[f][0]] + 2.f * best[f][1][pick[f][1]];
  }
  const int fb = nforms == 2 && step_ms[1] < step_ms[0] ? 1 : 0;
  c->stage_launch = forms[fb];
  c->plain_variant[0] = pick[fb][0];
  c->plain_variant[1] = pick[fb][1];
  c->launches += nl;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned[key] = Tuned{c->plain_variant[0], c->plain_variant[1], c->stage_launch};
  return IBM_OK;
}

static ibm_status capture_step_graph(ibm_case *c) {
  cudaGraph_t g = nullptr;
  CU(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  int nl = enqueue_step(c);
  cudaError_t e = cudaStreamEndCapture(c->stream, &g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(IBM_ECUDA, "step capture failed: %s", cudaGetErrorString(e));
  }
  e = cudaGraphInstantiate(&c->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    c->graph = nullptr;
    cudaGetLastError();
    return fail(IBM_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
  }
  c->graph_launches = nl;
  return IBM_OK;
}

extern "C" ibm_status ibm_step(ibm_case *c, int nsteps) {
  if (!c) return fail(IBM_EINVAL, "case is NULL");
  if (nsteps < 0) return fail(IBM_EINVAL, "nsteps < 0");
  if (nsteps == 0) return IBM_OK;
  if (!c->classified) {
    // the first classification runs outside any graph so that a static body's
    // graph holds only the flow kernels
    ibm_status r = do_classify(c);
    if (r != IBM_OK) return r;
  }
  if (fused_cfl(c) && !c->dt_valid) {
    // first step (or state replaced): dt from the current state; afterwards
    // every step's last stage provides the next dt
    int nl = 0;
    launch_dt_f32(c->k, c->M, c->tag, c->ds, c->stream, &nl);
    c->launches += nl;
    c->dt_valid = true;
  }
  if (c->plain_variant[0] < 0 && !persistent_step(c)) {
    ibm_status r = tune_plain_variant(c);
    if (r != IBM_OK) return r;
  }
  if (c->use_graphs && !c->profiling) {
    if (!c->graph) {
      ibm_status r = capture_step_graph(c);
      if (r != IBM_OK) return r;
    }
    for (int n = 0; n < nsteps; n++) CU(cudaGraphLaunch(c->graph, c->stream));
    c->launches += (long long)nsteps * c->graph_launches;
  } else {
    for (int n = 0; n < nsteps; n++) c->launches += enqueue_step(c);
  }
  CU(cudaGetLastError());
  return IBM_OK;
}

namespace ibm {

// batched groups run the explicit stages only: dual time and bodies moving under the fluid force (whose
// steps add the force and the body update) advance on their own streams
bool case_batchable(const ibm_case *c) {
  // dual-time groups are compiled for WENO5 and the linear reconstruction only
  return c->precision == IBM_PREC_FP32_BULK && !(c->k.dual && (c->k.tvd2 || c->k.quad));
}

int case_variant(const ibm_case *c) { return (c->k.tvd2 ? 1 : 0) | (c->k.quad ? 2 : 0); }

int case_subiters(const ibm_case *c) { return c->k.dual ? c->k.subiters : 0; }

bool case_coupled(const ibm_case *c) { return c->k.motion.kind == IBM_MOTION_COUPLED; }

ibm_status case_prepare_batch(ibm_case *c) {
  if (!c->classified) {
    ibm_status r = do_classify(c);
    if (r != IBM_OK) return r;
  }
  if (fused_cfl(c) && !c->dt_valid) {
    int nl = 0;
    launch_dt_f32(c->k, c->M, c->tag, c->ds, c->stream, &nl);
    c->launches += nl;
    c->dt_valid = true;
  }
  CU(cudaGetLastError());
  return IBM_OK;
}

int case_enqueue_prestage(ibm_case *c) {
  int nl = 0;
  bool geo_open = false;  // as in enqueue_step: the stencils (and force) overlap the rest, joined at the end
  if (c->k.motion.kind != IBM_MOTION_STATIC) {
    const long long before = c->launches;
    geo_open = c->sb != nullptr;
    do_classify(c, geo_open);
    nl += (int)(c->launches - before);
    c->launches = before;
  }
  if (c->k.dual) {  // as in a dual-time step of the case alone: W^{n-1} <- W^n <- W and the BDF part
    launch_dual_levels(c->k, c->A, c->Wn, c->G, c->ds, c->stream);
    nl += 1;
  } else {
    if (c->k.motion.kind == IBM_MOTION_COUPLED) nl += enqueue_force(c);  // Eq. 10: the force at the step's start
    if (!fused_cfl(c)) launch_dt_f32(c->k, c->M, c->tag, c->ds, c->stream, &nl);
  }
  geometry_join(c);
  if (geo_open) prof_mark(c, 4, false);
  return nl;
}

int case_enqueue_poststage(ibm_case *c) {
  if (c->k.dual) {
    launch_dual_end(c->k, c->ds, c->stream);
    return 1;
  }
  if (c->k.motion.kind == IBM_MOTION_COUPLED) {  // Eq. 10: position and velocity over the step
    launch_body_end(c->ds, c->stream);
    return 1;
  }
  return 0;
}

void case_stage_desc(const ibm_case *c, StageCase *out) {
  fill_stage_case(c->k, c->M, c->F1, c->F2, c->A, c->tag, c->sid, c->rst, c->tile_body, c->body_tiles, c->body_cap,
                  c->ds, fused_cfl(c), out);
  out->rsq = c->rsq;
  if (c->k.dual) {
    out->B = c->B;
    out->C = c->C;
    out->G = c->G;
    out->Q0 = c->Q0;
  }
}

cudaStream_t case_stream(const ibm_case *c) { return c->stream; }

void case_add_launches(ibm_case *c, long long n) { c->launches += n; }

}  // namespace ibm

extern "C" ibm_status ibm_autotune(ibm_case *c, int enable) {
  if (!c) return fail(IBM_EINVAL, "case is NULL");
  if (c->graph) return fail(IBM_ESTATE, "ibm_autotune: the case has already stepped");
  c->autotune = enable != 0;
  c->plain_variant[0] = c->plain_variant[1] = -1;
  return IBM_OK;
}

extern "C" ibm_status ibm_use_tma(ibm_case *c, int enable) {
  if (!c) return fail(IBM_EINVAL, "case is NULL");
  if (c->graph) {  // the captured step holds the old choice
    CU(cudaStreamSynchronize(c->stream));
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  c->use_tma = enable != 0;
  return IBM_OK;
}

extern "C" ibm_status ibm_use_persistent(ibm_case *c, int enable) {
  if (!c) return fail(IBM_EINVAL, "case is NULL");
  if (c->graph) {  // the captured step holds the old choice
    CU(cudaStreamSynchronize(c->stream));
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  c->use_persist = enable != 0;
  return IBM_OK;
}

extern "C" ibm_status ibm_stage_launches(ibm_case *c, int mode) {
  if (!c) return fail(IBM_EINVAL, "case is NULL");
  if (mode < 0 || mode > 2) return fail(IBM_EINVAL, "mode must be 0, 1 or 2");
  if (c->graph) {  // the captured step holds the old choice
    CU(cudaStreamSynchronize(c->stream));
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  if ((mode > 0) != (c->stage_launch > 0)) c->plain_variant[0] = c->plain_variant[1] = -1;  // other kernels: retune
  c->stage_launch = mode;
  c->launch_pinned = true;
  return IBM_OK;
}

extern "C" ibm_status ibm_persistent_grid(ibm_case *c, int blocks) {
  if (!c) return fail(IBM_EINVAL, "case is NULL");
  if (blocks < 0) return fail(IBM_EINVAL, "blocks < 0");
  if (c->graph) {
    CU(cudaStreamSynchronize(c->stream));
    cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
  }
  c->step_grid = blocks > 0 ? std::min(blocks, step_f32_grid(c->k, c->step_variant)) : 0;
  return IBM_OK;
}

extern "C" ibm_status ibm_check_float_conversions(uint64_t *checked, uint64_t *mismatched) {
  if (!checked || !mismatched) return fail(IBM_EINVAL, "ibm_check_float_conversions: NULL output");
  unsigned long long n = 0, bad = 0;
  const cudaError_t e = check_float_conversions(&n, &bad);
  if (e != cudaSuccess) return fail(IBM_ECUDA, "conversion check failed: %s", cudaGetErrorString(e));
  *checked = n;
  *mismatched = bad;
  return IBM_OK;
}

extern "C" ibm_status ibm_use_graphs(ibm_case *c, int enable) {
  if (!c) return fail(IBM_EINVAL, "case is NULL");
  c->use_graphs = enable != 0;
  return IBM_OK;
}

extern "C" ibm_status ibm_profile_enable(ibm_case *c, int enable) {
  if (!c) return fail(IBM_EINVAL, "case is NULL");
  if (enable && !c->ev[0]) {
    for (int q = 0; q < ibm_case::NEV; q++) CU(cudaEventCreate(&c->ev[q]));
  }
  c->profiling = enable != 0;
  return IBM_OK;
}

extern "C" ibm_status ibm_profile_read(ibm_case *c, double *ms, int64_t *launches, int n_groups) {
  if (!c || !ms || !launches || n_groups < 0 || n_groups > ibm_case::NGROUP)
    return fail(IBM_EINVAL, "bad arguments");
  CU(cudaStreamSynchronize(c->stream));
  for (int g = 0; g < n_groups; g++) {
    ms[g] = 0.0;
    launches[g] = 0;
  }
  for (int q = 0; q + 1 < c->nev; q += 2) {
    int g = c->ev_group[q / 2];
    float t = 0.f;
    CU(cudaEventElapsedTime(&t, c->ev[q], c->ev[q + 1]));
    if (g < n_groups) {
      ms[g] += t;
      launches[g] += 1;
    }
  }
  bool over = c->ev_overflow;
  c->nev = 0;
  c->ev_overflow = false;
  if (over) return fail(IBM_ESTATE, "profiling record overflowed; read more often");
  return IBM_OK;
}

static ibm_status sync_and_check(ibm_case *c) {
  CU(cudaMemcpyAsync(c->hds, c->ds, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  if (c->hds->err & ERR_CAPACITY)
    return fail(IBM_ECAPACITY, "IB/ghost list overflow: %d nodes, capacity %d", c->hds->offset[4], c->cap);
  if (c->hds->err & ERR_STENCIL) return fail(IBM_ESTENCIL, "an IB/ghost node found no valid interpolation corner");
  if (c->hds->err & ERR_TIMEOUT) return fail(IBM_ECUDA, "a bounded device wait for a TMA tile copy gave up");
  return IBM_OK;
}

extern "C" ibm_status ibm_sync(ibm_case *c) {
  if (!c) return fail(IBM_EINVAL, "case is NULL");
  return sync_and_check(c);
}

// copy between a [4][ny][nx] host/device buffer and the padded state planes
static ibm_status copy_state(ibm_case *c, double *dst, const double *src, bool to_user, bool user_on_device) {
  const Consts &k = c->k;
  double *base = c->A;
  if (to_user && c->precision == IBM_PREC_FP32_BULK) {
    // the FP64 state holds dU; hand out absolute conserved variables
    if (!c->stage64) CU(cudaMallocAsync((void **)&c->stage64, 4 * (size_t)k.plane * sizeof(double), c->stream));
    launch_pert_to_abs64(k, c->A, c->stage64, c->stream);
    c->launches++;
    base = c->stage64;
  }
  cudaMemcpyKind kind = to_user ? (user_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost)
                                : (user_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice);
  for (int v = 0; v < 4; v++) {
    double *dev = (to_user ? base : c->A) + v * k.plane + cidx(k, 0, 0);
    double *usr = (to_user ? dst : (double *)src) + (size_t)v * k.nx * k.ny;
    if (to_user)
      CU(cudaMemcpy2DAsync(usr, sizeof(double) * k.nx, dev, sizeof(double) * k.pitch, sizeof(double) * k.nx, k.ny,
                           kind, c->stream));
    else
      CU(cudaMemcpy2DAsync(dev, sizeof(double) * k.pitch, usr, sizeof(double) * k.nx, sizeof(double) * k.nx, k.ny,
                           kind, c->stream));
  }
  return IBM_OK;
}

extern "C" ibm_status ibm_get_state(ibm_case *c, int what, void *dst, size_t bytes, int dst_on_device) {
  if (!c || !dst) return fail(IBM_EINVAL, "case or dst is NULL");
  const Consts &k = c->k;
  const size_t ncell = (size_t)k.nx * k.ny;
  ibm_status r = sync_and_check(c);
  if (r != IBM_OK && r != IBM_ECAPACITY && r != IBM_ESTENCIL) return r;
  const DevState &h = *c->hds;
  cudaMemcpyKind d2x = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  switch (what) {
    case IBM_STATE_FP64:
      if (bytes < 4 * ncell * sizeof(double)) return fail(IBM_EINVAL, "dst too small");
      {
        ibm_status q = copy_state(c, (double *)dst, nullptr, true, dst_on_device);
        if (q != IBM_OK) return q;
      }
      break;
    case IBM_TAGS:
      if (bytes < ncell) return fail(IBM_EINVAL, "dst too small");
      CU(cudaMemcpyAsync(dst, c->tag, ncell, d2x, c->stream));
      break;
    case IBM_LIST_COUNTS:
      if (bytes < 4 * sizeof(int32_t)) return fail(IBM_EINVAL, "dst too small");
      if (dst_on_device)
        CU(cudaMemcpyAsync(dst, c->ds->count, 4 * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->stream));
      else
        std::memcpy(dst, h.count, 4 * sizeof(int32_t));
      break;
    case IBM_STENCILS: {
      size_t n = (size_t)(h.offset[4] < c->cap ? h.offset[4] : c->cap);
      if (bytes < n * sizeof(ibm_stencil)) return fail(IBM_EINVAL, "dst too small for %zu stencils", n);
      if (n) CU(cudaMemcpyAsync(dst, c->st, n * sizeof(ibm_stencil), d2x, c->stream));
      break;
    }
    case IBM_TIME: {
      if (bytes < 2 * sizeof(double)) return fail(IBM_EINVAL, "dst too small");
      double tt[2] = {h.t, h.dt};
      if (dst_on_device) {
        CU(cudaMemcpyAsync(dst, tt, sizeof tt, cudaMemcpyHostToDevice, c->stream));
        CU(cudaStreamSynchronize(c->stream));
      } else std::memcpy(dst, tt, sizeof tt);
      break;
    }
    case IBM_STEPS: {
      if (bytes < sizeof(int64_t)) return fail(IBM_EINVAL, "dst too small");
      int64_t n = h.steps;
      if (dst_on_device) {
        CU(cudaMemcpyAsync(dst, &n, sizeof n, cudaMemcpyHostToDevice, c->stream));
        CU(cudaStreamSynchronize(c->stream));
      } else std::memcpy(dst, &n, sizeof n);
      break;
    }
    case IBM_TUNING: {
      if (bytes < 2 * sizeof(int32_t) || dst_on_device)
        return fail(IBM_EINVAL, "IBM_TUNING: host int32[2] destination");
      const int32_t v[2] = {c->plain_variant[0], c->plain_variant[1]};
      std::memcpy(dst, v, sizeof v);
      break;
    }
    case IBM_STAGE_LAUNCH: {
      if (bytes < sizeof(int32_t) || dst_on_device) return fail(IBM_EINVAL, "IBM_STAGE_LAUNCH: host int32 destination");
      const int32_t v = c->precision == IBM_PREC_FP32_BULK ? c->stage_launch : -1;
      std::memcpy(dst, &v, sizeof v);
      break;
    }
    case IBM_BODY: {
      if (bytes < 6 * sizeof(double)) return fail(IBM_EINVAL, "dst too small");
      const double b[6] = {h.bX[0], h.bX[1], h.bV[0], h.bV[1], h.bF[0], h.bF[1]};
      if (dst_on_device) {
        CU(cudaMemcpyAsync(dst, b, sizeof b, cudaMemcpyHostToDevice, c->stream));
        CU(cudaStreamSynchronize(c->stream));
      } else std::memcpy(dst, b, sizeof b);
      break;
    }
    default:
      return fail(IBM_EINVAL, "unknown quantity %d", what);
  }
  CU(cudaStreamSynchronize(c->stream));
  return r;
}

static ibm_status set_state(ibm_case *c, const void *src, size_t bytes, int src_on_device, bool wait_for_host) {
  if (!c || !src) return fail(IBM_EINVAL, "case or src is NULL");
  const size_t ncell = (size_t)c->k.nx * c->k.ny;
  if (bytes < 4 * ncell * sizeof(double)) return fail(IBM_EINVAL, "src too small");
  // one contiguous copy into a device staging buffer (the full bandwidth of the host link, where a pitched copy
  // into the padded layout moves row by row), then one kernel: layout, perturbation form and FP32 mirror
  if (!c->stage64) CU(cudaMallocAsync((void **)&c->stage64, 4 * (size_t)c->k.plane * sizeof(double), c->stream));
  CU(cudaMemcpyAsync(c->stage64, src, 4 * ncell * sizeof(double),
                     src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
  launch_set_state(c->k, c->stage64, c->A, c->M, c->stream);
  c->launches += 1;
  if (c->M) c->dt_valid = false;
  if (!src_on_device && wait_for_host) CU(cudaStreamSynchronize(c->stream));
  CU(cudaGetLastError());
  return IBM_OK;
}

extern "C" ibm_status ibm_set_state(ibm_case *c, const void *src, size_t bytes, int src_on_device) {
  return set_state(c, src, bytes, src_on_device, true);
}

extern "C" ibm_status ibm_set_state_async(ibm_case *c, const void *src, size_t bytes, int src_on_device) {
  return set_state(c, src, bytes, src_on_device, false);
}

extern "C" ibm_status ibm_forces(ibm_case *c, double out[4]) {
  if (!c || !out) return fail(IBM_EINVAL, "case or out is NULL");
  if (c->g.nv <= 0) {
    for (int q = 0; q < 4; q++) out[q] = 0.0;
    return IBM_OK;
  }
  if (!c->classified) {
    ibm_status r = do_classify(c);
    if (r != IBM_OK) return r;
  }
  launch_forces_f64(c->k, c->g, c->tag, c->A, c->precision == IBM_PREC_FP32_BULK, c->ds, c->stream);
  c->launches++;
  ibm_status r = sync_and_check(c);
  for (int q = 0; q < 4; q++) out[q] = c->hds->force[q];
  return r;
}

extern "C" ibm_status ibm_surface(ibm_case *c, double *cp, double *cf, int nseg) {
  if (!c || !cp || !cf) return fail(IBM_EINVAL, "case or output is NULL");
  if (nseg != c->g.nv) return fail(IBM_EINVAL, "nseg %d differs from the body's %d segments", nseg, c->g.nv);
  if (c->g.nv <= 0) return IBM_OK;
  if (!c->classified) {
    ibm_status r = do_classify(c);
    if (r != IBM_OK) return r;
  }
  launch_forces_f64(c->k, c->g, c->tag, c->A, c->precision == IBM_PREC_FP32_BULK, c->ds, c->stream, false, c->surf);
  c->launches++;
  CU(cudaMemcpyAsync(cp, c->surf, (size_t)nseg * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaMemcpyAsync(cf, c->surf + nseg, (size_t)nseg * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  return sync_and_check(c);
}

extern "C" ibm_status ibm_destroy_case(ibm_case *c) {
  if (!c) return IBM_OK;
  cudaStreamSynchronize(c->stream);
  free_case(c);
  return IBM_OK;
}

extern "C" int64_t ibm_launch_count(const ibm_case *c) { return c ? c->launches : 0; }

extern "C" const char *ibm_last_error(void) { return g_err; }

extern "C" ibm_status ibm__noalloc_fail(ibm_status s, const char *msg) { return fail(s, "%s", msg); }
