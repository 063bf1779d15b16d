// Immersed-boundary geometry kernels: body pose, ray-casting classification,
// IB / ghost tagging with ordered list compaction, closest features,
// pseudo-normals, boundary points, probe / image points, interpolation
// stencils, and the surface force integral.
//
// This translation unit is compiled with -fmad=false: every floating-point
// result here is a sequence of IEEE binary64 basic operations (and sqrt) with
// no contraction, so tags, lists and stencils are reproducible bit for bit by
// any IEEE implementation that performs the same operations in the same
// order.  No transcendental function is used on these paths.
#include <math_constants.h>
#include <mutex>

#include <algorithm>

#include "ibm_internal.cuh"

namespace ibm {

// ---------------------------------------------------------------------------
// Sec. 4.2: pseudo-normals.  Segment k of the CCW polyline runs from vertex k
// to k+1; its outward normal is the travel direction turned clockwise.  The
// 2-D vertex pseudo-normal weights its two incident segments equally (each
// incident "face" enters Eq. 2 / Eq. 3 with the same weight) and is
// normalised.  The vertex also gets the local curvature of the supersonic
// moving-body condition (Eq. 7): the signed Menger curvature of its two
// incident segments, 2 (e1 x e2) / (|e1| |e2| |e1 + e2|), positive for a left
// (convex) turn of the CCW polyline (1/r exactly on a regular polygon
// inscribed in a circle of radius r).  One thread per vertex.
// ---------------------------------------------------------------------------
__global__ void k_normals(int nv, const double *__restrict__ v, double *snx, double *sny, double *vnx,
                          double *vny, double *vk) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nv) return;
  int k1 = (k + 1 == nv) ? 0 : k + 1;
  int km = (k == 0) ? nv - 1 : k - 1;
  // own segment normal
  double ex = v[2 * k1] - v[2 * k], ey = v[2 * k1 + 1] - v[2 * k + 1];
  double L = sqrt(ex * ex + ey * ey);
  double nx = ey / L, ny = -ex / L;
  snx[k] = nx;
  sny[k] = ny;
  // previous segment normal (recomputed with the same operations)
  double fx = v[2 * k] - v[2 * km], fy = v[2 * k + 1] - v[2 * km + 1];
  double Lm = sqrt(fx * fx + fy * fy);
  double mx = fy / Lm, my = -fx / Lm;
  double sx = mx + nx, sy = my + ny;
  double S = sqrt(sx * sx + sy * sy);
  if (S > 0.0) {
    vnx[k] = sx / S;
    vny[k] = sy / S;
  } else {
    vnx[k] = nx;
    vny[k] = ny;
  }
  // curvature: e1 = previous segment (fx, fy), e2 = own segment (ex, ey)
  double cx = fx + ex, cy = fy + ey;
  double L3 = sqrt(cx * cx + cy * cy);
  double den = Lm * L * L3;
  vk[k] = den > 0.0 ? 2.0 * (fx * ey - fy * ex) / den : 0.0;
}

void launch_normals(int nv, const double *v, double *snx, double *sny, double *vnx, double *vny, double *vk,
                    cudaStream_t s) {
  if (nv <= 0) return;
  k_normals<<<(nv + 127) / 128, 128, 0, s>>>(nv, v, snx, sny, vnx, vny, vk);
}

// Pose of vertex v: the reference vertex shifted by the translation X, or for a pitching body (Sec. 7.2) turned
// about the pivot by the body angle whose cosine and sine are cs, sn.
__device__ __forceinline__ void pose_vertex(const Consts &k, const Geom &g, int v, const double X[2], double cs,
                                            double sn, double &x, double &y) {
  if (k.motion.kind == IBM_MOTION_PITCH) {
    const double rx = g.vref[2 * v] - k.motion.pivot[0], ry = g.vref[2 * v + 1] - k.motion.pivot[1];
    x = k.motion.pivot[0] + (cs * rx - sn * ry);
    y = k.motion.pivot[1] + (sn * rx + cs * ry);
  } else {
    x = g.vref[2 * v] + X[0];
    y = g.vref[2 * v + 1] + X[1];
  }
}

// a pitching body's segment and vertex normals: the reference pose's, turned with the body
__device__ __forceinline__ void pose_normals(const Geom &g, int v, double cs, double sn) {
  g.snx[v] = cs * g.rsnx[v] - sn * g.rsny[v];
  g.sny[v] = sn * g.rsnx[v] + cs * g.rsny[v];
  g.vnx[v] = cs * g.rvnx[v] - sn * g.rvny[v];
  g.vny[v] = sn * g.rvnx[v] + cs * g.rvny[v];
}

// translation X and, for a pitching body, cos / sin of the body angle at the start of the step
__device__ __forceinline__ void pose_params(const Consts &k, const DevState *ds, double X[2], double &cs,
                                            double &sn) {
  double V[2], A[2];
  body_motion(k, ds, ds->t, X, V, A);
  cs = 1.0;
  sn = 0.0;
  if (k.motion.kind == IBM_MOTION_PITCH) {
    double th, om, al;
    pitch_at(k.motion, ds->t, &th, &om, &al);
    sincos(th, &sn, &cs);
  }
}

// ---------------------------------------------------------------------------
// Body pose at the start of the step (prescribed translation or pitching) and
// its axis-aligned bounding box.  One block.
// ---------------------------------------------------------------------------
__global__ void k_pose(Consts k, Geom g, DevState *ds) {
  __shared__ double X[2], rot[2];
  if (threadIdx.x == 0) {
    double P[2];
    pose_params(k, ds, P, rot[0], rot[1]);
    X[0] = P[0];
    X[1] = P[1];
    ds->pos[0] = P[0];
    ds->pos[1] = P[1];
  }
  __syncthreads();
  // each thread keeps the extremes of its own vertices; then warp and block reductions (min / max are exact)
  double b[4] = {INFINITY, -INFINITY, INFINITY, -INFINITY};
  for (int v = threadIdx.x; v < g.nv; v += blockDim.x) {
    double x, y;
    pose_vertex(k, g, v, X, rot[0], rot[1], x, y);
    g.vx[v] = x;
    g.vy[v] = y;
    if (k.motion.kind == IBM_MOTION_PITCH) pose_normals(g, v, rot[0], rot[1]);
    b[0] = fmin(b[0], x);
    b[1] = fmax(b[1], x);
    b[2] = fmin(b[2], y);
    b[3] = fmax(b[3], y);
  }
  for (int off = 16; off > 0; off >>= 1) {
    b[0] = fmin(b[0], __shfl_xor_sync(0xffffffffu, b[0], off));
    b[1] = fmax(b[1], __shfl_xor_sync(0xffffffffu, b[1], off));
    b[2] = fmin(b[2], __shfl_xor_sync(0xffffffffu, b[2], off));
    b[3] = fmax(b[3], __shfl_xor_sync(0xffffffffu, b[3], off));
  }
  __shared__ double wb[32][4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0)
    for (int q = 0; q < 4; q++) wb[warp][q] = b[q];
  __syncthreads();  // (also orders this block's pose writes before the segment bounds read them)
  for (int v = threadIdx.x; v < g.nv; v += blockDim.x) {
    const int v1 = v + 1 == g.nv ? 0 : v + 1;
    segment_bound(g.vx[v], g.vy[v], g.vx[v1], g.vy[v1], g.sb + 3 * v);
  }
  if (threadIdx.x == 0) {
    for (int w = 1; w < nw; w++) {
      b[0] = fmin(b[0], wb[w][0]);
      b[1] = fmax(b[1], wb[w][1]);
      b[2] = fmin(b[2], wb[w][2]);
      b[3] = fmax(b[3], wb[w][3]);
    }
    for (int q = 0; q < 4; q++) ds->bbox[q] = b[q];
    ds->bcell[0] = (int)floor((b[0] - k.x0) / k.dx - 0.5) - 3;
    ds->bcell[1] = (int)ceil((b[1] - k.x0) / k.dx - 0.5) + 3;
    ds->bcell[2] = (int)floor((b[2] - k.y0) / k.dy - 0.5) - 3;
    ds->bcell[3] = (int)ceil((b[3] - k.y0) / k.dy - 0.5) + 3;
  }
}

void launch_pose(const Consts &k, const Geom &g, DevState *ds, cudaStream_t s) {
  k_pose<<<1, 256, 0, s>>>(k, g, ds);
}

// ---------------------------------------------------------------------------
// Sec. 3.2: ray-casting classification of cell centres.  Ray along +x; the
// segment A->B is crossed iff (A.y > P.y) != (B.y > P.y) and the crossing
// abscissa A.x + (P.y-A.y)(B.x-A.x)/(B.y-A.y) lies strictly right of P; odd
// parity = solid.  Centres outside the axis-aligned bounding box are fluid
// (all cells are cleared first).  One warp per cell inside the box: the lanes
// split the segments and the crossing parity is the XOR over lanes.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_classify(Consts k, Geom g, uint8_t *__restrict__ solid,
                                                  const DevState *__restrict__ ds, int maxw, int maxh) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const double b0 = ds->bbox[0], b1 = ds->bbox[1], b2 = ds->bbox[2], b3 = ds->bbox[3];
  // cell range covering the box: centres x0 + (i + 1/2) dx in [b0, b1]
  const int ilo = max(0, (int)floor((b0 - k.x0) / k.dx - 0.5) - 1);
  const int jlo = max(0, (int)floor((b2 - k.y0) / k.dy - 0.5) - 1);
  if (warp >= maxw * maxh) return;
  const int i = ilo + warp % maxw, j = jlo + warp / maxw;
  if (i >= k.nx || j >= k.ny) return;
  const double px = k.x0 + ((double)i + 0.5) * k.dx;
  const double py = k.y0 + ((double)j + 0.5) * k.dy;
  if (px < b0 || px > b1 || py < b2 || py > b3) return;  // stays fluid
  int odd = 0;
  for (int e = lane; e < g.nv; e += 32) {
    const int e1 = (e + 1 == g.nv) ? 0 : e + 1;
    const double ax = g.vx[e], ay = g.vy[e], bx = g.vx[e1], by = g.vy[e1];
    if ((ay > py) != (by > py)) {
      double t1 = py - ay;
      double t2 = bx - ax;
      double t3 = by - ay;
      double xint = ax + (t1 * t2) / t3;
      if (xint > px) odd ^= 1;
    }
  }
  odd = __popc(__ballot_sync(0xffffffffu, odd)) & 1;
  if (lane == 0) solid[j * k.nx + i] = (uint8_t)odd;
}

void launch_classify(const Consts &k, const Geom &g, uint8_t *solid, const DevState *ds, int maxw, int maxh,
                     cudaStream_t s) {
  const int ncell = k.nx * k.ny;
  cudaMemsetAsync(solid, 0, (size_t)ncell, s);
  if (g.nv <= 0 || maxw <= 0 || maxh <= 0) return;
  const long long warps = (long long)maxw * maxh;
  k_classify<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(k, g, solid, ds, maxw, maxh);
}

// ---------------------------------------------------------------------------
// Sec. 3.2 + Sec. 5: tags and ordered lists.
//  IB  : fluid cell with a solid 4-neighbour.
//  Gk  : solid cell whose nearest non-solid cell along a grid line is k = 1, 2
//        or 3 cells away (three ghost layers for WENO5).
// Lists are compacted in row-major cell order: per-block counts by warp
// ballots, one-block scan of the block counts, then a ballot-ranked scatter.
// ---------------------------------------------------------------------------
constexpr int TAG_BLOCK = 1024;

__device__ inline uint8_t tag_of(const Consts &k, const uint8_t *__restrict__ solid, int i, int j) {
  const int nx = k.nx, ny = k.ny;
  if (!solid[j * nx + i]) {
    bool ib = (i + 1 < nx && solid[j * nx + i + 1]) || (i > 0 && solid[j * nx + i - 1]) ||
              (j + 1 < ny && solid[(j + 1) * nx + i]) || (j > 0 && solid[(j - 1) * nx + i]);
    return ib ? IB : FLUID;
  }
  for (int d = 1; d <= 3; d++) {
    if ((i + d < nx && !solid[j * nx + i + d]) || (i - d >= 0 && !solid[j * nx + i - d]) ||
        (j + d < ny && !solid[(j + d) * nx + i]) || (j - d >= 0 && !solid[(j - d) * nx + i]))
      return (uint8_t)(G1 + d - 1);
  }
  return SOLID;
}

__device__ inline int list_kind(uint8_t t) {  // -1: not listed; 0 IB; 1..3 G1..G3
  return t == IB ? 0 : (t >= G1 ? (int)t - G1 + 1 : -1);
}

__global__ void __launch_bounds__(TAG_BLOCK) k_tag_count(Consts k, const uint8_t *__restrict__ solid,
                                                         uint8_t *__restrict__ tag, int *__restrict__ blockcounts) {
  __shared__ int wc[TAG_BLOCK / 32][4];
  const int n = blockIdx.x * TAG_BLOCK + threadIdx.x;
  const int ncell = k.nx * k.ny;
  int kind = -1;
  if (n < ncell) {
    uint8_t t = tag_of(k, solid, n % k.nx, n / k.nx);
    tag[n] = t;
    kind = list_kind(t);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = 0; q < 4; q++) {
    unsigned m = __ballot_sync(0xffffffffu, kind == q);
    if (lane == 0) wc[warp][q] = __popc(m);
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    int s = 0;
    for (int w = 0; w < TAG_BLOCK / 32; w++) s += wc[w][threadIdx.x];
    blockcounts[blockIdx.x * 4 + threadIdx.x] = s;
  }
}

// exclusive scan of per-block counts for each kind (in place), totals and
// kind offsets into the concatenated list (IB, G1, G2, G3)
__global__ void __launch_bounds__(1024) k_scan_blocks(int nblk, int *blockcounts, DevState *ds, int cap) {
  __shared__ int wsum[32][4];
  __shared__ int tot[4];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int per = (nblk + 1023) / 1024;
  const int b0 = tid * per, b1 = min(nblk, b0 + per);
  int s[4] = {0, 0, 0, 0};
  for (int b = b0; b < b1; b++)
    for (int q = 0; q < 4; q++) s[q] += blockcounts[b * 4 + q];
  // inclusive scan of the 1024 partial sums: within each warp by shuffles, then over the 32 warp totals
  int inc[4];
  for (int q = 0; q < 4; q++) {
    inc[q] = s[q];
    for (int off = 1; off < 32; off <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, inc[q], off);
      if (lane >= off) inc[q] += v;
    }
  }
  if (lane == 31)
    for (int q = 0; q < 4; q++) wsum[warp][q] = inc[q];
  __syncthreads();
  if (warp == 0) {
    for (int q = 0; q < 4; q++) {
      int w = wsum[lane][q];
      for (int off = 1; off < 32; off <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, w, off);
        if (lane >= off) w += v;
      }
      wsum[lane][q] = w;  // inclusive over warps
      if (lane == 31) tot[q] = w;
    }
  }
  __syncthreads();
  int run[4];
  for (int q = 0; q < 4; q++) run[q] = inc[q] - s[q] + (warp > 0 ? wsum[warp - 1][q] : 0);
  for (int b = b0; b < b1; b++)
    for (int q = 0; q < 4; q++) {
      int c = blockcounts[b * 4 + q];
      blockcounts[b * 4 + q] = run[q];
      run[q] += c;
    }
  if (tid == 0) {
    int off = 0;
    for (int q = 0; q < 4; q++) {
      ds->count[q] = tot[q];
      ds->offset[q] = off;
      off += tot[q];
    }
    ds->offset[4] = off;
    if (off > cap) ds->err |= ERR_CAPACITY;
  }
}

__global__ void __launch_bounds__(TAG_BLOCK) k_scatter(Consts k, const uint8_t *__restrict__ tag,
                                                       const int *__restrict__ blockoff, const DevState *ds,
                                                       ibm_stencil *__restrict__ st, int cap) {
  __shared__ int wc[TAG_BLOCK / 32][4];
  const int n = blockIdx.x * TAG_BLOCK + threadIdx.x;
  const int ncell = k.nx * k.ny;
  const int kind = n < ncell ? list_kind(tag[n]) : -1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  int rank = 0;
  for (int q = 0; q < 4; q++) {
    unsigned m = __ballot_sync(0xffffffffu, kind == q);
    if (lane == 0) wc[warp][q] = __popc(m);
    if (kind == q) rank = __popc(m & lt);
  }
  __syncthreads();
  if (kind >= 0) {
    int before = 0;
    for (int w = 0; w < warp; w++) before += wc[w][kind];
    int pos = ds->offset[kind] + blockoff[blockIdx.x * 4 + kind] + before + rank;
    if (pos < cap) {
      st[pos].cell = n;
      st[pos].kind = kind;
    }
  }
}

void launch_tags(const Consts &k, const uint8_t *solid, uint8_t *tag, int *blockcounts, DevState *ds, int cap,
                 ibm_stencil *st, cudaStream_t s, int *nlaunch) {
  const int ncell = k.nx * k.ny;
  const int nblk = (ncell + TAG_BLOCK - 1) / TAG_BLOCK;
  k_tag_count<<<nblk, TAG_BLOCK, 0, s>>>(k, solid, tag, blockcounts);
  k_scan_blocks<<<1, 1024, 0, s>>>(nblk, blockcounts, ds, cap);
  k_scatter<<<nblk, TAG_BLOCK, 0, s>>>(k, tag, blockcounts, ds, st, cap);
  *nlaunch += 3;
}

// Sec. 4.6 / Sec. 5: interpolation square around (X, Y); bilinear when all
// four corners carry an allowed tag, inverse-distance (1/r^2) weights over
// the allowed corners otherwise, all weight on a corner hit exactly.
__device__ int interp_square(const Consts &k, const uint8_t *__restrict__ tag, double X, double Y,
                             unsigned allowed, int *i0o, int *j0o, double w[4]) {
  double gx = (X - k.x0) / k.dx - 0.5;
  double gy = (Y - k.y0) / k.dy - 0.5;
  int i0 = (int)floor(gx), j0 = (int)floor(gy);
  int mask = 0;
  for (int q = 0; q < 4; q++) {
    int ci = i0 + (q & 1), cj = j0 + (q >> 1);
    w[q] = 0.0;
    if (ci < 0 || ci >= k.nx || cj < 0 || cj >= k.ny) continue;
    if (allowed & (1u << tag[cj * k.nx + ci])) mask |= 1 << q;
  }
  *i0o = i0;
  *j0o = j0;
  if (mask == 15) {
    double xc0 = k.x0 + ((double)i0 + 0.5) * k.dx;
    double yc0 = k.y0 + ((double)j0 + 0.5) * k.dy;
    double fx = (X - xc0) / k.dx;
    double fy = (Y - yc0) / k.dy;
    w[0] = (1.0 - fx) * (1.0 - fy);
    w[1] = fx * (1.0 - fy);
    w[2] = (1.0 - fx) * fy;
    w[3] = fx * fy;
  } else if (mask != 0) {
    double inv[4] = {0.0, 0.0, 0.0, 0.0};
    int hit = -1;
    for (int q = 0; q < 4 && hit < 0; q++) {
      if (!(mask >> q & 1)) continue;
      double xk = k.x0 + ((double)(i0 + (q & 1)) + 0.5) * k.dx;
      double yk = k.y0 + ((double)(j0 + (q >> 1)) + 0.5) * k.dy;
      double rx = X - xk, ry = Y - yk;
      double r2 = rx * rx + ry * ry;
      if (r2 == 0.0) hit = q;
      else inv[q] = 1.0 / r2;
    }
    if (hit >= 0) {
      w[hit] = 1.0;
    } else {
      double s = 0.0;
      for (int q = 0; q < 4; q++)
        if (mask >> q & 1) s += inv[q];
      for (int q = 0; q < 4; q++)
        if (mask >> q & 1) w[q] = inv[q] / s;
    }
  }
  return mask;
}

constexpr unsigned ALLOW_FLUID = 1u << FLUID;
constexpr unsigned ALLOW_FLUID_IB = (1u << FLUID) | (1u << IB);

// Sec. 4.1: the point of segment kk nearest (px, py) -- a vertex (region VERTEX, feature the vertex) or the
// foot point (region FACE, feature the segment) -- and its squared distance
__device__ __forceinline__ double seg_closest(const Geom &g, int kk, double px, double py, double *cxo, double *cyo,
                                              int *fo, int *ro) {
  const int k1 = (kk + 1 == g.nv) ? 0 : kk + 1;
  const double ax = g.vx[kk], ay = g.vy[kk], bx = g.vx[k1], by = g.vy[k1];
  const double ex = bx - ax, ey = by - ay;
  const double wx = px - ax, wy = py - ay;
  const double num = wx * ex + wy * ey;
  const double den = ex * ex + ey * ey;
  double cx, cy;
  if (num <= 0.0) {
    cx = ax; cy = ay; *fo = kk; *ro = IBM_REGION_VERTEX;
  } else if (num >= den) {
    cx = bx; cy = by; *fo = k1; *ro = IBM_REGION_VERTEX;
  } else {
    const double t = num / den;
    cx = ax + t * ex; cy = ay + t * ey; *fo = kk; *ro = IBM_REGION_FACE;
  }
  *cxo = cx;
  *cyo = cy;
  const double ddx = px - cx, ddy = py - cy;
  return ddx * ddx + ddy * ddy;
}

// Sec. 4.3: crossing of the line through (px, py) along (nx, ny) with segment kk, at parameter u on the
// segment and signed distance sv along the normal, on the side the node's kind allows (a ghost node, inside
// the body, finds the wall along the normal, sv >= 0; an IB node, in the fluid, against it, sv <= 0); false if
// there is none
__device__ __forceinline__ bool seg_crossing(const Geom &g, int kk, double px, double py, double nx, double ny,
                                             bool ghost, double *uo, double *svo) {
  const int k1 = (kk + 1 == g.nv) ? 0 : kk + 1;
  const double ax = g.vx[kk], ay = g.vy[kk];
  const double ex = g.vx[k1] - ax, ey = g.vy[k1] - ay;
  const double den = ex * ny - ey * nx;
  if (den == 0.0) return false;
  const double wx = px - ax, wy = py - ay;
  const double u = (wx * ny - wy * nx) / den;
  if (u < 0.0 || u > 1.0) return false;
  const double sv = (wx * ey - wy * ex) / den;
  if (ghost ? (sv < 0.0) : (sv > 0.0)) return false;
  *uo = u;
  *svo = sv;
  return true;
}

// quadratic form (Sec. 4.5, Sec. 5): the second probe / image point one diagonal spacing beyond the first, on the
// same corner set and pushed out the same way while its square has no usable corner (kept out of line: it is
// compiled into every stencil kernel, most of whose cases take the linear form)
static __device__ __noinline__ void second_probe(const Consts &k, const uint8_t *__restrict__ tag, double bx,
                                                 double by, double nx, double ny, double xi_probe, unsigned allowed,
                                                 ibm_stencil &s) {
  double xi2 = xi_probe + k.h;
  int ib = 0, jb = 0, maskb = 0, nstepb = 0;
  for (;;) {
    double X = bx + xi2 * nx, Y = by + xi2 * ny;
    maskb = interp_square(k, tag, X, Y, allowed, &ib, &jb, s.wb);
    if (maskb != 0 || nstepb == 3) break;
    xi2 = xi2 + k.dmin;
    nstepb++;
  }
  s.i0b = ib;
  s.j0b = jb;
  s.maskb = maskb;
  s.nstepb = nstepb;
  s.xi_probe2 = xi2;
}

// the FP32 quadratic part of a record (out of line, like second_probe)
static __device__ __noinline__ void write_quad_stencil(const Consts &k, const ibm_stencil &s, RStencilQ *out) {
  *out = quad_stencil(k, s);
}

// The rest of one node's stencil once the closest feature (feat, region, foot point cc) and the boundary point
// search (found_abs < inf: signed distance bsv at parameter bsu on segment bsg) are known: boundary point,
// image / probe distance, interpolation square (Sec. 4.3-4.6), curvature at P' (Eq. 7); writes the record,
// and with rs its compact FP32 form and the cell -> stencil map.
__device__ __forceinline__ void stencil_tail(const Consts &k, const Geom &g, const uint8_t *__restrict__ tag,
                                             DevState *ds, int e, double px, double py,
                                             int feat, int region, double ccx, double ccy, double found_abs,
                                             double bsv, double bsu, int bsg, double nx, double ny,
                                             ibm_stencil *__restrict__ st, RStencil32 *__restrict__ rs,
                                             int *__restrict__ sid) {
  ibm_stencil s = st[e];  // the list entry: cell and kind
  const int kind = s.kind;
  const bool ghost = kind > 0;
  const int nv = g.nv;
  double bx, by, xi_node;
  int fb;
  if (found_abs < INFINITY) {
    bx = px + bsv * nx;
    by = py + bsv * ny;
    xi_node = -bsv;
    fb = 0;
  } else {
    const double ddx = px - ccx, ddy = py - ccy;
    const double d = sqrt(ddx * ddx + ddy * ddy);
    bx = ccx;
    by = ccy;
    xi_node = ghost ? -d : d;
    fb = 1;
  }
  double xi_probe;
  if (kind == 0) {
    xi_probe = xi_node + k.h;
  } else {
    xi_probe = -xi_node;
    if (xi_probe < 0.5 * k.dmin) xi_probe = 0.5 * k.dmin;
  }
  const unsigned allowed = kind == 0 ? ALLOW_FLUID : ALLOW_FLUID_IB;
  int i0 = 0, j0 = 0, mask = 0, nstep = 0;
  double w[4];
  for (;;) {
    double X = bx + xi_probe * nx, Y = by + xi_probe * ny;
    mask = interp_square(k, tag, X, Y, allowed, &i0, &j0, w);
    if (mask != 0 || nstep == 3) break;
    xi_probe = xi_probe + k.dmin;
    nstep++;
  }
  if (mask == 0) atomicOr(&ds->err, ERR_STENCIL);
  // curvature at P' (Eq. 7): linear between the end-vertex curvatures of the segment holding P', or the
  // vertex curvature when P' falls back to a closest vertex
  double curv;
  if (fb && region == IBM_REGION_VERTEX) {
    curv = g.vk[feat];
  } else {
    int sg = bsg;
    double uu = bsu;
    if (fb) {  // P' is the foot point on segment feat
      const int f1 = (feat + 1 == nv) ? 0 : feat + 1;
      const double ex = g.vx[f1] - g.vx[feat], ey = g.vy[f1] - g.vy[feat];
      sg = feat;
      uu = ((ccx - g.vx[feat]) * ex + (ccy - g.vy[feat]) * ey) / (ex * ex + ey * ey);
    }
    const int s1 = (sg + 1 == nv) ? 0 : sg + 1;
    curv = (1.0 - uu) * g.vk[sg] + uu * g.vk[s1];
  }
  s.curv = curv;
  s.feature = feat;
  s.region = fb ? IBM_REGION_FALLBACK : region;
  s.i0 = i0;
  s.j0 = j0;
  s.mask = mask;
  s.nstep = nstep;
  s.nx = nx;
  s.ny = ny;
  s.bx = bx;
  s.by = by;
  s.xi_node = xi_node;
  s.xi_probe = xi_probe;
  for (int q = 0; q < 4; q++) s.w[q] = w[q];
  // quadratic form (Sec. 4.5, Sec. 5): the second probe / image point one diagonal spacing beyond the first, on the
  // same corner set and pushed out the same way while its square has no usable corner
  s.i0b = s.j0b = s.maskb = s.nstepb = 0;
  s.xi_probe2 = 0.0;
  for (int q = 0; q < 4; q++) s.wb[q] = 0.0;
  if (k.quad && mask != 0) second_probe(k, tag, bx, by, nx, ny, xi_probe, allowed, s);
  st[e] = s;
  if (rs) {
    RStencil32 r;
    r.cell = (int)cidx(k, s.cell % k.nx, s.cell / k.nx);
    r.corner = s.mask ? (int)cidx(k, s.i0, s.j0) : 0;
    r.ccell = s.mask ? s.j0 * k.nx + s.i0 : 0;
    r.mask = s.mask | (s.kind == 0 ? 16 : 0);  // bit 4: IB node
    r.ratio = (float)(s.xi_node / s.xi_probe);
    r.dxi = (float)(s.xi_probe - s.xi_node);
    r.nx = (float)s.nx;
    r.ny = (float)s.ny;
    for (int q = 0; q < 4; q++) r.w[q] = (float)s.w[q];
    r.curv = (float)s.curv;
    const bool pitching = k.motion.kind == IBM_MOTION_PITCH;  // P' relative to the pivot (wall motion)
    r.rx = pitching ? (float)(s.bx - k.motion.pivot[0]) : 0.f;
    r.ry = pitching ? (float)(s.by - k.motion.pivot[1]) : 0.f;
    rs[e] = r;
    sid[s.cell] = e;
    if (g.rsq) write_quad_stencil(k, s, g.rsq + e);
  }
}

// Sec. 4.1-4.6, Sec. 5: one stencil per listed node, a group of NL lanes
// per node (blocks striding over the list).  The lanes
// split the segments of the two searches (closest feature, boundary point);
// the group keeps the (distance, segment) lexicographic minimum, which is the
// first minimum of a sequential scan.
// rs / sid (optional): the FP32 compact form of each stencil and the cell ->
// stencil map of the FP32-bulk reconstruction.
// Pruning (bodies of up to STENCIL_PRUNE_MAX vertices): every segment's
// bounding circle in FP32 (centre, half length plus a margin of 1e-5 of the
// coordinates' size, far above FP32 rounding) bounds the distance from the
// node to the segment from below and above; a segment whose lower bound
// exceeds the smallest upper bound cannot hold the closest point, and one
// whose lower bound exceeds the |s| of a crossing already found cannot hold a
// nearer boundary point (the crossing lies on the segment).  The searches run
// the exact FP64 tests on the others only, so the result is the exhaustive
// search's, bit for bit.
constexpr int STENCIL_PRUNE_MAX = 2048;

// Lanes per listed node: a whole warp, or half a warp (two nodes per warp).  Half a warp splits a node's
// segments about as well (its candidates after pruning are a few neighbouring segments), and the FP64 work
// that follows the searches, on the group's first lane, then shares its warp instructions with the other
// node's: fewer FP64 warp instructions per node, which bounds the kernel when many nodes fill the GPU; with
// few nodes the kernel is bound by one node's latency, which a whole warp keeps shorter.

// group_argmin over aligned groups of NL lanes: the lane holding the (value, index) lexicographic minimum
template <int NL>
__device__ __forceinline__ int group_argmin(double v, int idx) {
  int src = threadIdx.x & 31;
  for (int off = NL / 2; off > 0; off >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, off);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, off);
    const int os = __shfl_xor_sync(0xffffffffu, src, off);
    if (ov < v || (ov == v && oi < idx)) {
      v = ov;
      idx = oi;
      src = os;
    }
  }
  return src;
}

template <int NL>
__global__ void __launch_bounds__(128) k_stencils(Consts k, Geom g, const uint8_t *__restrict__ tag,
                                                  ibm_stencil *__restrict__ st, int cap, DevState *ds,
                                                  RStencil32 *__restrict__ rs, int *__restrict__ sid) {
  constexpr int STENCIL_NODES = 128 / NL;  // nodes per block in flight
  extern __shared__ float s_sb[];  // per segment: centre x, y and bounding radius, FP32 (segment_bound)
  const int total = min(ds->offset[4], cap);
  const int nv = g.nv;
  const bool prune = nv <= STENCIL_PRUNE_MAX;
  const int lane = threadIdx.x & 31, gl = lane % NL;
  if ((int)blockIdx.x * STENCIL_NODES >= total) return;
  if (prune) {  // the pose kernel's segment bounds of this pose
    for (int kk = threadIdx.x; kk < 3 * nv; kk += 128) s_sb[kk] = g.sb[kk];
    __syncthreads();
  }
  // NL lanes per listed node splitting the segments of the searches; the loop runs alike for the whole warp
  // (every lane takes part in the shuffles), a group past the end of the list idle inside it
  for (int e0 = (int)blockIdx.x * STENCIL_NODES + (int)(threadIdx.x >> 5) * (32 / NL); e0 < total;
       e0 += (int)gridDim.x * STENCIL_NODES) {
    const int e = e0 + lane / NL;
    const bool act = e < total;
    const int cell = act ? st[e].cell : 0, kind = act ? st[e].kind : 0;
    const int i = cell % k.nx, j = cell / k.nx;
    const double px = k.x0 + ((double)i + 0.5) * k.dx;
    const double py = k.y0 + ((double)j + 0.5) * k.dy;
    const float pxf = (float)px, pyf = (float)py;
    // the smallest upper bound of the node's distance to a segment
    float ub = INFINITY;
    if (prune && act) {
      for (int kk = gl; kk < nv; kk += NL) {
        const float dx = pxf - s_sb[3 * kk], dy = pyf - s_sb[3 * kk + 1];
        ub = fminf(ub, sqrtf(dx * dx + dy * dy) + s_sb[3 * kk + 2]);
      }
    }
    for (int o = NL / 2; o > 0; o >>= 1) ub = fminf(ub, __shfl_xor_sync(0xffffffffu, ub, o));
    // closest feature (Sec. 4.1)
    double best = INFINITY, bcx = 0.0, bcy = 0.0;
    int bseg = 0x7fffffff, bfeat = 0, breg = 0;
    if (act) {
      for (int kk = gl; kk < nv; kk += NL) {
        if (prune) {
          const float dx = pxf - s_sb[3 * kk], dy = pyf - s_sb[3 * kk + 1];
          if (sqrtf(dx * dx + dy * dy) - s_sb[3 * kk + 2] > ub) continue;
        }
        double cx, cy;
        int f, r;
        const double d2 = seg_closest(g, kk, px, py, &cx, &cy, &f, &r);
        if (d2 < best) {
          best = d2; bseg = kk; bfeat = f; breg = r; bcx = cx; bcy = cy;
        }
      }
    }
    int win = group_argmin<NL>(best, bseg);
    const int feat = __shfl_sync(0xffffffffu, bfeat, win);
    const int region = __shfl_sync(0xffffffffu, breg, win);
    const double ccx = __shfl_sync(0xffffffffu, bcx, win), ccy = __shfl_sync(0xffffffffu, bcy, win);
    double nx = 0.0, ny = 0.0;
    if (act) {
      if (region == IBM_REGION_FACE) {
        nx = g.snx[feat];
        ny = g.sny[feat];
      } else {
        nx = g.vnx[feat];
        ny = g.vny[feat];
      }
    }
    // boundary point on the line along the local normal (Sec. 4.3): first the segments that can hold the
    // closest point, then, beyond them, those that can hold a crossing no farther than the best found (all of
    // them if none was found)
    const bool ghost = kind > 0;
    double bs_best = INFINITY, bs_s = 0.0, bs_u = 0.0;
    int bs_seg = 0x7fffffff;
    float bound = INFINITY;
    for (int pass = 0; pass < (prune ? 2 : 1); pass++) {
      if (pass == 1) {
        const int w2 = group_argmin<NL>(bs_best, bs_seg);
        const double found = __shfl_sync(0xffffffffu, bs_best, w2);
        bound = found < INFINITY ? (float)found * (1.f + 1e-6f) : INFINITY;
      }
      if (!act) continue;
      for (int kk = gl; kk < nv; kk += NL) {
        if (prune) {
          const float dx = pxf - s_sb[3 * kk], dy = pyf - s_sb[3 * kk + 1];
          const float lb = sqrtf(dx * dx + dy * dy) - s_sb[3 * kk + 2];
          if (pass == 0 ? lb > ub : (lb <= ub || lb > bound)) continue;
        }
        double u, sv;
        if (!seg_crossing(g, kk, px, py, nx, ny, ghost, &u, &sv)) continue;
        const double as = fabs(sv);
        if (as < bs_best || (as == bs_best && kk < bs_seg)) {
          bs_best = as; bs_s = sv; bs_u = u; bs_seg = kk;
        }
      }
    }
    win = group_argmin<NL>(bs_best, bs_seg);
    const double found_abs = __shfl_sync(0xffffffffu, bs_best, win);
    const double bsv = __shfl_sync(0xffffffffu, bs_s, win);
    const double bsu = __shfl_sync(0xffffffffu, bs_u, win);
    const int bsg = __shfl_sync(0xffffffffu, bs_seg, win);
    if (act && gl == 0)
      stencil_tail(k, g, tag, ds, e, px, py, feat, region, ccx, ccy, found_abs, bsv, bsu, bsg, nx, ny, st, rs,
                   sid);
    __syncwarp();
  }
}

// stencils of the listed nodes: 128 / lanes per node per 128-thread block, blocks striding over the list
static void launch_stencil_kernel(const Consts &k, const Geom &g, const uint8_t *tag, ibm_stencil *st, int cap,
                                  DevState *ds, RStencil32 *rs, int *sid, cudaStream_t s) {
  if (cap <= 0) return;
  const size_t smem = g.nv <= STENCIL_PRUNE_MAX ? 3 * sizeof(float) * g.nv : 0;
  if (g.stencil_lanes == 16)
    k_stencils<16><<<(unsigned)min((cap + 7) / 8, 8 * 152), 128, smem, s>>>(k, g, tag, st, cap, ds, rs, sid);
  else
    k_stencils<32><<<(unsigned)min((cap + 3) / 4, 8 * 152), 128, smem, s>>>(k, g, tag, st, cap, ds, rs, sid);
}

// ---------------------------------------------------------------------------
// Fused per-classification geometry for bodies of up to FUSED_MAX_VERTS
// vertices (see launch_fused_geometry).
// ---------------------------------------------------------------------------

constexpr int ROW_XMAX = 64;  // crossings of one row kept in shared memory by the fused classification

// clipped cell rectangle [ilo, ihi] x [jlo, jhi]; empty if ilo > ihi or jlo > jhi
__device__ __forceinline__ void clip_rect(const Consts &k, int r[4]) {
  r[0] = max(r[0], 0);
  r[1] = min(r[1], k.nx - 1);
  r[2] = max(r[2], 0);
  r[3] = min(r[3], k.ny - 1);
}

// (1) pose + ray-parity classification of the cells of urect = (current
// bounding-box cells, 3-cell margin) united with the previous rectangle.
// Every block poses the vertices into shared memory and reduces the box
// itself (exact operations, identical in every block); block 0 publishes
// them.  One warp per cell, grid-stride over the rectangle.
__global__ void __launch_bounds__(256) k_pose_classify(Consts k, Geom g, uint8_t *__restrict__ solid,
                                                       DevState *ds) {
  extern __shared__ double sv[];  // x[nv] then y[nv]
  __shared__ double X[2], rot[2];
  __shared__ double wb[8][4];
  __shared__ double bb[4];
  __shared__ int rect[4];
  const int nv = g.nv;
  if (threadIdx.x == 0) {
    double P[2];
    pose_params(k, ds, P, rot[0], rot[1]);
    X[0] = P[0];
    X[1] = P[1];
  }
  __syncthreads();
  double b[4] = {INFINITY, -INFINITY, INFINITY, -INFINITY};
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    double x, y;
    pose_vertex(k, g, v, X, rot[0], rot[1], x, y);
    sv[v] = x;
    sv[nv + v] = y;
    if (blockIdx.x == 0) {
      g.vx[v] = x;
      g.vy[v] = y;
      if (k.motion.kind == IBM_MOTION_PITCH) pose_normals(g, v, rot[0], rot[1]);
    }
    b[0] = fmin(b[0], x);
    b[1] = fmax(b[1], x);
    b[2] = fmin(b[2], y);
    b[3] = fmax(b[3], y);
  }
  for (int off = 16; off > 0; off >>= 1) {
    b[0] = fmin(b[0], __shfl_xor_sync(0xffffffffu, b[0], off));
    b[1] = fmax(b[1], __shfl_xor_sync(0xffffffffu, b[1], off));
    b[2] = fmin(b[2], __shfl_xor_sync(0xffffffffu, b[2], off));
    b[3] = fmax(b[3], __shfl_xor_sync(0xffffffffu, b[3], off));
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0)
    for (int q = 0; q < 4; q++) wb[warp][q] = b[q];
  __syncthreads();
  if (blockIdx.x == 0)  // the stencil searches' segment bounds of this pose
    for (int v = threadIdx.x; v < nv; v += blockDim.x) {
      const int v1 = v + 1 == nv ? 0 : v + 1;
      segment_bound(sv[v], sv[nv + v], sv[v1], sv[nv + v1], g.sb + 3 * v);
    }
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; w++) {
      b[0] = fmin(b[0], wb[w][0]);
      b[1] = fmax(b[1], wb[w][1]);
      b[2] = fmin(b[2], wb[w][2]);
      b[3] = fmax(b[3], wb[w][3]);
    }
    int bc[4];
    bc[0] = (int)floor((b[0] - k.x0) / k.dx - 0.5) - 3;
    bc[1] = (int)ceil((b[1] - k.x0) / k.dx - 0.5) + 3;
    bc[2] = (int)floor((b[2] - k.y0) / k.dy - 0.5) - 3;
    bc[3] = (int)ceil((b[3] - k.y0) / k.dy - 0.5) + 3;
    int r[4] = {bc[0], bc[1], bc[2], bc[3]};
    clip_rect(k, r);
    if (ds->prect_valid) {
      const bool empty = r[0] > r[1] || r[2] > r[3];
      const int *p = ds->prect;
      if (p[0] <= p[1] && p[2] <= p[3]) {
        if (empty) {
          for (int q = 0; q < 4; q++) r[q] = p[q];
        } else {
          r[0] = min(r[0], p[0]);
          r[1] = max(r[1], p[1]);
          r[2] = min(r[2], p[2]);
          r[3] = max(r[3], p[3]);
        }
      }
    }
    for (int q = 0; q < 4; q++) {
      bb[q] = b[q];
      rect[q] = r[q];
    }
    if (blockIdx.x == 0) {
      ds->pos[0] = X[0];
      ds->pos[1] = X[1];
      for (int q = 0; q < 4; q++) {
        ds->bbox[q] = b[q];
        ds->bcell[q] = bc[q];
        ds->urect[q] = r[q];
      }
    }
  }
  __syncthreads();
  if (rect[0] > rect[1] || rect[2] > rect[3]) return;
  const int W = rect[1] - rect[0] + 1, H = rect[3] - rect[2] + 1;
  const double b0 = bb[0], b1 = bb[1], b2 = bb[2], b3 = bb[3];
  const int nwarps = (int)gridDim.x * (blockDim.x >> 5);
  // one warp per row of the rectangle: a segment's crossing abscissa depends only on the row's ordinate, so
  // the lanes find the crossings of the row once (the same operations as a per-cell test, hence the same bits)
  // and every cell of the row counts those right of its centre; a row with more than ROW_XMAX crossings
  // falls back to testing every segment per cell
  __shared__ double xs[8][ROW_XMAX];
  for (int r = (int)blockIdx.x * (blockDim.x >> 5) + warp; r < H; r += nwarps) {
    const int j = rect[2] + r;
    const double py = k.y0 + ((double)j + 0.5) * k.dy;
    int nx_ = 0;  // crossings of the row found so far (warp-uniform)
    bool overflow = false;
    const bool row_in = !(py < b2 || py > b3);
    if (row_in) {
      for (int e0 = 0; e0 < nv; e0 += 32) {
        const int e = e0 + lane;
        bool cross = false;
        double xint = 0.0;
        if (e < nv) {
          const int e1 = (e + 1 == nv) ? 0 : e + 1;
          const double ax = sv[e], ay = sv[nv + e], bx = sv[e1], by = sv[nv + e1];
          if ((ay > py) != (by > py)) {
            double t1 = py - ay;
            double t2 = bx - ax;
            double t3 = by - ay;
            xint = ax + (t1 * t2) / t3;
            cross = true;
          }
        }
        const unsigned m = __ballot_sync(0xffffffffu, cross);
        const int pos = nx_ + __popc(m & ((1u << lane) - 1u));
        if (cross && pos < ROW_XMAX) xs[warp][pos] = xint;
        nx_ += __popc(m);
      }
      overflow = nx_ > ROW_XMAX;
    }
    __syncwarp();
    for (int i = rect[0] + lane; i <= rect[1]; i += 32) {
      const double px = k.x0 + ((double)i + 0.5) * k.dx;
      int odd = 0;
      if (row_in && !(px < b0 || px > b1)) {
        if (!overflow) {
          for (int q = 0; q < nx_; q++) odd ^= xs[warp][q] > px ? 1 : 0;
        } else {
          for (int e = 0; e < nv; e++) {
            const int e1 = (e + 1 == nv) ? 0 : e + 1;
            const double ax = sv[e], ay = sv[nv + e], bx = sv[e1], by = sv[nv + e1];
            if ((ay > py) != (by > py)) {
              double t1 = py - ay;
              double t2 = bx - ax;
              double t3 = by - ay;
              double xint = ax + (t1 * t2) / t3;
              if (xint > px) odd ^= 1;
            }
          }
        }
      }
      solid[j * k.nx + i] = (uint8_t)odd;
    }
    __syncwarp();
  }
  (void)W;
}

// does the tile's loaded range [lo, hi] (before domain mapping) along one axis
// reach the cells [blo, bhi]?  (A periodic side that the range crosses wraps
// it: yes.)
__device__ __forceinline__ bool tile_axis_reaches(int lo, int hi, int n, int bc_lo, int bc_hi, int blo, int bhi) {
  if ((lo < 0 && bc_lo == IBM_BC_PERIODIC) || (hi >= n && bc_hi == IBM_BC_PERIODIC)) return true;
  lo = max(lo, 0);
  hi = min(hi, n - 1);
  return lo <= bhi && hi >= blo;
}

// tag rule of tag_of on a staged copy of the solid flags: rows ey0.., columns
// ex0.. of width ew (the rectangle plus the 3-cell reach of the rule)
__device__ __forceinline__ uint8_t tag_of_staged(const Consts &k, const uint8_t *ss, int ex0, int ey0, int ew, int i,
                                                 int j) {
  const int nx = k.nx, ny = k.ny;
#define SOL(ii, jj) ss[((jj)-ey0) * ew + ((ii)-ex0)]
  if (!SOL(i, j)) {
    bool ib = (i + 1 < nx && SOL(i + 1, j)) || (i > 0 && SOL(i - 1, j)) || (j + 1 < ny && SOL(i, j + 1)) ||
              (j > 0 && SOL(i, j - 1));
    return ib ? IB : FLUID;
  }
  for (int d = 1; d <= 3; d++) {
    if ((i + d < nx && !SOL(i + d, j)) || (i - d >= 0 && !SOL(i - d, j)) || (j + d < ny && !SOL(i, j + d)) ||
        (j - d >= 0 && !SOL(i, j - d)))
      return (uint8_t)(G1 + d - 1);
  }
#undef SOL
  return SOLID;
}

// (2) one block of 1024 threads over urect: tags (and sid reset), the
// row-major IB / G1-G3 lists, then the body-tile flags of every stage tile and
// their ascending list.  Rectangles of up to staged_cap cells (with the rule's
// 3-cell reach; dynamic shared memory sized from the body's pose-independent
// box) work on shared-memory copies of the solid flags and tags; cells
// outside urect are fluid (invariant), so no other tag is read.  The lists
// are ranked with one block-wide scan: every thread owns a contiguous chunk of
// the rectangle (row-major), counts its nodes per class, takes its offsets
// from an exclusive scan of the counts and writes its nodes in order.  Ends by
// recording the current rectangle for the next classification.
constexpr int STAGED_CELLS_MAX = 100 * 1024;  // 200 KB of shared memory for the two staged byte arrays
__global__ void __launch_bounds__(1024) k_tags_lists(Consts k, const uint8_t *__restrict__ solid,
                                                     uint8_t *__restrict__ tag, int *__restrict__ sid,
                                                     ibm_stencil *__restrict__ st, int cap,
                                                     uint8_t *__restrict__ tile_body, int *__restrict__ body_tiles,
                                                     int body_cap, DevState *ds, int staged_cap) {
  extern __shared__ uint8_t s_dyn[];
  uint8_t *s_sol = s_dyn, *s_tag = s_dyn + staged_cap;
  __shared__ int wc[32][4];
  __shared__ int tot[4], run[4], off[4];
  __shared__ int wsum[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r0 = ds->urect[0], r1 = ds->urect[1], r2 = ds->urect[2], r3 = ds->urect[3];
  const int W = r0 <= r1 && r2 <= r3 ? r1 - r0 + 1 : 0, H = W ? r3 - r2 + 1 : 0;
  const int n = W * H;
  const int ex0 = max(r0 - 3, 0), ex1 = min(r1 + 3, k.nx - 1), ey0 = max(r2 - 3, 0), ey1 = min(r3 + 3, k.ny - 1);
  const int ew = ex1 - ex0 + 1, eh = ey1 - ey0 + 1;
  const bool staged = n > 0 && ew * eh <= staged_cap && n <= staged_cap;
  if (staged)
    for (int m = tid; m < ew * eh; m += 1024) s_sol[m] = solid[(ey0 + m / ew) * k.nx + ex0 + m % ew];
  __syncthreads();
  // pass 1: tags, counts per kind
  int cnt[4] = {0, 0, 0, 0};
  for (int m = tid; m < n; m += 1024) {
    const int i = r0 + m % W, j = r2 + m / W;
    const uint8_t t = staged ? tag_of_staged(k, s_sol, ex0, ey0, ew, i, j) : tag_of(k, solid, i, j);
    tag[j * k.nx + i] = t;
    if (staged) s_tag[m] = t;
    if (sid) sid[j * k.nx + i] = -1;
    const int q = list_kind(t);
    if (q >= 0) cnt[q]++;
  }
  for (int q = 0; q < 4; q++) {
    int v = cnt[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) wc[warp][q] = v;
  }
  __syncthreads();
  if (tid < 4) {
    int v = 0;
    for (int w = 0; w < 32; w++) v += wc[w][tid];
    tot[tid] = v;
    run[tid] = 0;
  }
  __syncthreads();
  if (tid == 0) {
    int o = 0;
    for (int q = 0; q < 4; q++) {
      off[q] = o;
      ds->count[q] = tot[q];
      ds->offset[q] = o;
      o += tot[q];
    }
    ds->offset[4] = o;
    if (o > cap) atomicOr(&ds->err, ERR_CAPACITY);
  }
  __syncthreads();
  // pass 2: every thread owns the contiguous chunk [m0, m1) of the rectangle (row-major); its nodes of each
  // class follow those of the threads before it
  const int chunk = (n + 1023) / 1024, m0 = min(n, tid * chunk), m1 = min(n, m0 + chunk);
  int own[4] = {0, 0, 0, 0};
  for (int m = m0; m < m1; m++) {
    const int q = list_kind(staged ? s_tag[m] : tag[(r2 + m / W) * k.nx + r0 + m % W]);
    if (q >= 0) own[q]++;
  }
  // exclusive scan of the four counts over the block: within the warp by shuffles, then over the warp totals
  int before[4];
  for (int q = 0; q < 4; q++) {
    int v = own[q];
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    before[q] = v - own[q];
    if (lane == 31) wc[warp][q] = v;
  }
  __syncthreads();
  if (tid < 4) {  // exclusive scan of the warp totals of class tid (32 values)
    int acc = 0;
    for (int w = 0; w < 32; w++) {
      const int x = wc[w][tid];
      wc[w][tid] = acc;
      acc += x;
    }
  }
  __syncthreads();
  int pos[4];
  for (int q = 0; q < 4; q++) pos[q] = off[q] + wc[warp][q] + before[q];
  for (int m = m0; m < m1; m++) {
    const int i = r0 + m % W, j = r2 + m / W, cell = j * k.nx + i;
    const int q = list_kind(staged ? s_tag[m] : tag[cell]);
    if (q < 0) continue;
    const int p_ = pos[q]++;
    if (p_ < cap) {
      st[p_].cell = cell;
      st[p_].kind = q;
    }
  }
  (void)run;
  __syncthreads();
  // body-tile flags (one warp per tile; tiles out of reach of the body's cells skipped) and their list
  if (tile_body) {
    constexpr int T = STAGE_TILE, HX = T + 2 * NG, HY = T + 2 * NG;
    const int ntx = (k.nx + T - 1) / T, nt = ntx * ((k.ny + T - 1) / T);
    const int nty = (k.ny + T - 1) / T;
    const int bl = ds->bcell[0], bh = ds->bcell[1], cl = ds->bcell[2], ch = ds->bcell[3];
    for (int t = tid; t < nt; t += 1024) tile_body[t] = 0;
    __syncthreads();
    // tiles whose loaded range can reach the body's cells: a conservative range of tile columns and rows
    // (every tile along an axis whose sides are periodic), then the exact test
    int tx0 = 0, tx1 = ntx - 1, ty0 = 0, ty1 = nty - 1;
    if (k.bc[0] != IBM_BC_PERIODIC && k.bc[1] != IBM_BC_PERIODIC) {
      tx0 = max(0, (max(bl, 0) - NG) / T - 1);
      tx1 = min(ntx - 1, (min(bh, k.nx - 1) + NG) / T + 1);
    }
    if (k.bc[2] != IBM_BC_PERIODIC && k.bc[3] != IBM_BC_PERIODIC) {
      ty0 = max(0, (max(cl, 0) - NG) / T - 1);
      ty1 = min(nty - 1, (min(ch, k.ny - 1) + NG) / T + 1);
    }
    const int cw = tx1 - tx0 + 1, ncand = n > 0 && tx0 <= tx1 && ty0 <= ty1 ? cw * (ty1 - ty0 + 1) : 0;
    for (int c = warp; c < ncand; c += 32) {
      const int tx = tx0 + c % cw, ty = ty0 + c / cw;
      const int t = ty * ntx + tx, i0 = tx * T, j0 = ty * T;
      bool hit = false;
      if (tile_axis_reaches(i0 - NG, i0 + T + NG - 1, k.nx, k.bc[0], k.bc[1], bl, bh) &&
          tile_axis_reaches(j0 - NG, j0 + T + NG - 1, k.ny, k.bc[2], k.bc[3], cl, ch)) {
        for (int m = lane; m < HX * HY; m += 32) {
          int gi = i0 - NG + m % HX, gj = j0 - NG + m / HX;
          if (!halo_map(k, gi, gj)) continue;
          if (gi < r0 || gi > r1 || gj < r2 || gj > r3) continue;  // fluid outside the rectangle
          const uint8_t tg = staged ? s_tag[(gj - r2) * W + (gi - r0)] : tag[gj * k.nx + gi];
          hit |= (tg == IB || tg >= G1);
        }
        hit = __any_sync(0xffffffffu, hit);
      }
      if (lane == 0 && hit) tile_body[t] = 1;
    }
    __syncthreads();
    // ascending list of the flagged tiles: per-thread runs, warp-shuffle scan, scan of the warp totals
    const int per = (nt + 1023) / 1024;
    const int t0 = tid * per, t1 = min(nt, t0 + per);
    int c = 0;
    for (int t = t0; t < t1; t++) c += tile_body[t];
    int inc = c;
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += v;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      int w = wsum[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += v;
      }
      wsum[lane] = w;
    }
    __syncthreads();
    int pos = inc - c + (warp > 0 ? wsum[warp - 1] : 0);
    for (int t = t0; t < t1; t++)
      if (tile_body[t]) {
        if (pos < body_cap) body_tiles[pos] = t;
        pos++;
      }
    if (tid == 0) {
      const int total = wsum[31];
      ds->nbody_tiles = min(total, body_cap);
      if (total > body_cap) atomicOr(&ds->err, ERR_CAPACITY);
    }
  }
  if (tid == 0) {
    int r[4] = {ds->bcell[0], ds->bcell[1], ds->bcell[2], ds->bcell[3]};
    clip_rect(k, r);
    for (int q = 0; q < 4; q++) ds->prect[q] = r[q];
    ds->prect_valid = 1;
  }
}

// Bodies whose pose-independent box holds more than LARGE_RECT cells: the same tags and lists over many blocks.
// Chunk c of the rectangle is its cells [c TAG_BLOCK, (c + 1) TAG_BLOCK) in row-major order; one block per
// chunk (chunks past the rectangle count zero), then the block scan of launch_tags and a rectangle scatter; the
// body-tile flags and list follow with launch_tile_lists.
constexpr long long LARGE_RECT = 8192;
__global__ void __launch_bounds__(TAG_BLOCK) k_rect_tags(Consts k, const uint8_t *__restrict__ solid,
                                                         uint8_t *__restrict__ tag, int *__restrict__ sid,
                                                         int *__restrict__ blockcounts, const DevState *ds) {
  __shared__ int wc[TAG_BLOCK / 32][4];
  const int r0 = ds->urect[0], r1 = ds->urect[1], r2 = ds->urect[2], r3 = ds->urect[3];
  const int W = r0 <= r1 && r2 <= r3 ? r1 - r0 + 1 : 0, H = W ? r3 - r2 + 1 : 0;
  const int m = blockIdx.x * TAG_BLOCK + threadIdx.x;
  int kind = -1;
  if (m < W * H) {
    const int i = r0 + m % W, j = r2 + m / W;
    const uint8_t t = tag_of(k, solid, i, j);
    tag[j * k.nx + i] = t;
    if (sid) sid[j * k.nx + i] = -1;
    kind = list_kind(t);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = 0; q < 4; q++) {
    const unsigned b = __ballot_sync(0xffffffffu, kind == q);
    if (lane == 0) wc[warp][q] = __popc(b);
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    int v = 0;
    for (int w = 0; w < TAG_BLOCK / 32; w++) v += wc[w][threadIdx.x];
    blockcounts[4 * blockIdx.x + threadIdx.x] = v;
  }
}

__global__ void __launch_bounds__(TAG_BLOCK) k_rect_scatter(Consts k, const uint8_t *__restrict__ tag,
                                                            const int *__restrict__ blockoff, DevState *ds,
                                                            ibm_stencil *__restrict__ st, int cap) {
  __shared__ int wc[TAG_BLOCK / 32][4];
  const int r0 = ds->urect[0], r1 = ds->urect[1], r2 = ds->urect[2], r3 = ds->urect[3];
  const int W = r0 <= r1 && r2 <= r3 ? r1 - r0 + 1 : 0, H = W ? r3 - r2 + 1 : 0;
  const int m = blockIdx.x * TAG_BLOCK + threadIdx.x;
  int kind = -1, cell = 0;
  if (m < W * H) {
    cell = (r2 + m / W) * k.nx + r0 + m % W;
    kind = list_kind(tag[cell]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  int rank = 0;
  for (int q = 0; q < 4; q++) {
    const unsigned b = __ballot_sync(0xffffffffu, kind == q);
    if (lane == 0) wc[warp][q] = __popc(b);
    if (kind == q) rank = __popc(b & lt);
  }
  __syncthreads();
  if (kind >= 0) {
    int before = 0;
    for (int w = 0; w < warp; w++) before += wc[w][kind];
    const int pos = ds->offset[kind] + blockoff[blockIdx.x * 4 + kind] + before + rank;
    if (pos < cap) {
      st[pos].cell = cell;
      st[pos].kind = kind;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {  // the rectangle of this classification, for the next one
    int r[4] = {ds->bcell[0], ds->bcell[1], ds->bcell[2], ds->bcell[3]};
    clip_rect(k, r);
    for (int q = 0; q < 4; q++) ds->prect[q] = r[q];
    ds->prect_valid = 1;
  }
}

// opt the one-block tag / list kernel into the dynamic shared memory its staging uses (once per process and
// device, before any capture)
void prepare_geometry_kernels() {
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 || done[dev]) return;
  cudaFuncSetAttribute(k_tags_lists, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * STAGED_CELLS_MAX);
  done[dev] = true;
}

int launch_fused_geometry(const Consts &k, const Geom &g, uint8_t *solid, uint8_t *tag, ibm_stencil *st, int cap,
                          RStencil32 *rs, int *sid, uint8_t *tile_body, int *body_tiles, int body_cap, int maxw,
                          int maxh, DevState *ds, int *blockcounts, cudaStream_t s, cudaStream_t ss,
                          cudaEvent_t ev_tags) {
  // one warp per row of the classification rectangle (at most the body's pose-independent height, the previous
  // rectangle's and the margins)
  const long long warps = 2LL * (maxh + 8);
  const int blocks = (int)std::min<long long>(std::max<long long>((warps + 7) / 8, 1), 4096);
  k_pose_classify<<<blocks, 256, 2 * sizeof(double) * g.nv, s>>>(k, g, solid, ds);
  // staged copies of the rectangle (plus the tag rule's reach) in dynamic shared memory, sized for the body's
  // pose-independent box with room for one step's motion; larger rectangles read global memory
  const long long want = (long long)(maxw + 24) * (maxh + 24);
  const int staged_cap = (int)std::min<long long>(want, STAGED_CELLS_MAX);
  int nl = 2;
  const bool large = (long long)maxw * maxh > LARGE_RECT && blockcounts;
  if (large) {
    // one block per chunk of the grid's size (the block counts are sized for it), so that any rectangle is
    // covered; blocks past the rectangle exit at once
    const int nchunk = (int)(((long long)k.nx * k.ny + TAG_BLOCK - 1) / TAG_BLOCK);
    k_rect_tags<<<nchunk, TAG_BLOCK, 0, s>>>(k, solid, tag, sid, blockcounts, ds);
    k_scan_blocks<<<1, 1024, 0, s>>>(nchunk, blockcounts, ds, cap);
    k_rect_scatter<<<nchunk, TAG_BLOCK, 0, s>>>(k, tag, blockcounts, ds, st, cap);
    nl += 2;
  } else {
    k_tags_lists<<<1, 1024, 2 * (size_t)staged_cap, s>>>(k, solid, tag, sid, st, cap, tile_body, body_tiles,
                                                         body_cap, ds, staged_cap);
  }
  // the stencils need the tags and the ordered list only: with a side stream they run there, beside the tile
  // lists (and whatever the caller enqueues next on s until it joins ss)
  cudaStream_t sst = s;
  if (ss && ev_tags && cap > 0) {
    cudaEventRecord(ev_tags, s);
    cudaStreamWaitEvent(ss, ev_tags, 0);
    sst = ss;
  }
  if (cap > 0) {
    launch_stencil_kernel(k, g, tag, st, cap, ds, rs, sid, sst);
    nl++;
  }
  if (large && tile_body) {
    launch_tile_lists(k, tag, tile_body, body_tiles, body_cap, ds, true, s);
    nl += 2;
  }
  return nl;
}

void launch_stencils(const Consts &k, const Geom &g, const uint8_t *tag, ibm_stencil *st, int cap, DevState *ds,
                     cudaStream_t s) {
  launch_stencil_kernel(k, g, tag, st, cap, ds, nullptr, nullptr, s);
}

// ---------------------------------------------------------------------------
// Sec. 6, Eq. 9: force on the body, midpoint rule per segment; surface
// pressure and wall shear from a probe one diagonal spacing out along the
// segment normal (inverse-distance weighted, Sec. 4.6), the pressure carried
// to the wall by the reconstruction's wall condition (Eq. 6-8, curvature at
// the segment midpoint); free-stream pressure subtracted.
// ---------------------------------------------------------------------------
// Eq. 9 over the body's segments: four lanes per segment, each taking one corner of the probe's interpolation
// square (the corners' conversions to primitives are the longest part of a segment's work), summed in corner
// order by shuffles -- the values a single lane forms, a masked corner adding an exact zero.  The segment's
// geometry and wall terms run on all four lanes alike.  One-warp blocks of FORCE_THREADS / 4 segments, up to
// FORCE_BLOCKS blocks striding over longer bodies; each block sums its segments in a fixed shuffle-tree order
// into a partial, and the last block to finish adds the partials in block order, so the sum is deterministic.
constexpr int FORCE_THREADS = 32, FORCE_BLOCKS = 64, FORCE_SEGS = FORCE_THREADS / 4;
__global__ void __launch_bounds__(FORCE_THREADS) k_forces_f64(Consts k, Geom g, const uint8_t *__restrict__ tag,
                                                              const double *__restrict__ A, bool pert, DevState *ds,
                                                              bool set_accel, double *__restrict__ surf) {
  __shared__ bool last;
  __shared__ double part[2 * FORCE_BLOCKS];
  double V[2], Acc[2], X[2];
  body_motion(k, ds, ds->t, X, V, Acc);
  const bool sup = supersonic_motion(k, V);
  const int cq = threadIdx.x & 3, base = threadIdx.x & ~3;
  double sx = 0.0, sy = 0.0;
  // the loop's trip count is the same for the whole warp (every lane takes part in the shuffles)
  for (int e0 = blockIdx.x * FORCE_SEGS; e0 < g.nv; e0 += gridDim.x * FORCE_SEGS) {
    const int e = e0 + (threadIdx.x >> 2);
    const bool valid = e < g.nv;
    const int e1 = (e + 1 >= g.nv) ? 0 : e + 1;
    double L = 1.0, tx = 0.0, ty = 0.0, nx = 0.0, ny = 0.0, mx = 0.0, my = 0.0, xi = k.h, w[4];
    int i0 = 0, j0 = 0, mask = 0;
    if (valid) {
      const double ax = g.vx[e], ay = g.vy[e];
      const double ex = g.vx[e1] - ax, ey = g.vy[e1] - ay;
      L = sqrt(ex * ex + ey * ey);
      tx = ex / L;
      ty = ey / L;
      nx = ty;
      ny = -tx;
      mx = ax + 0.5 * ex;
      my = ay + 0.5 * ey;
      for (int stp = 0; stp <= 3; stp++) {
        mask = interp_square(k, tag, mx + xi * nx, my + xi * ny, ALLOW_FLUID, &i0, &j0, w);
        if (mask) break;
        if (stp < 3) xi = xi + k.dmin;
      }
    }
    // this lane's corner: w_q (p, u, v, T) at the corner's cell
    double t[4] = {0.0, 0.0, 0.0, 0.0};
    if (mask >> cq & 1) {
      const long long id = cidx(k, i0 + (cq & 1), j0 + (cq >> 1));
      double U0 = A[id], U1 = A[id + k.plane], U2 = A[id + 2 * k.plane], U3 = A[id + 3 * k.plane];
      if (pert) {  // perturbation state dU -> absolute conserved
        U3 = k.Uinf[3] + U3 + k.Hinf * U0;
        U0 = 1.0 + U0;
        U1 = k.Uinf[1] + U1;
        U2 = k.Uinf[2] + U2;
      }
      const double r = U0, u = U1 / r, v = U2 / r;
      const double pr = (k.gamma - 1.0) * (U3 - 0.5 * r * (u * u + v * v));
      const double T = pr / (r * k.R);
      const double wq = cq == 0 ? w[0] : cq == 1 ? w[1] : cq == 2 ? w[2] : w[3];
      t[0] = wq * pr;
      t[1] = wq * u;
      t[2] = wq * v;
      t[3] = wq * T;
    }
    double qp[4] = {0.0, 0.0, 0.0, 0.0};
    for (int q = 0; q < 4; q++)
      for (int m = 0; m < 4; m++) qp[m] += __shfl_sync(0xffffffffu, t[m], base + q);
    if (!valid) continue;
    if (!mask) {
      if (surf && cq == 0) surf[e] = surf[g.nv + e] = CUDART_NAN;
      continue;
    }
    // wall pressure: the probe's, carried to the surface by the wall condition of the reconstruction
    double Vs[2], As[2];
    wall_kin(k, ds->t, mx, my, V, Acc, Vs, As);  // the wall's motion at the segment midpoint
    double G = -(nx * As[0] + ny * As[1]);
    if (sup) {
      double ut = (qp[1] - Vs[0]) * tx + (qp[2] - Vs[1]) * ty;
      G = G + ut * ut * (0.5 * (g.vk[e] + g.vk[e1]));
    }
    const double ps = qp[0] * exp(-xi * G / (k.R * qp[3]));
    const double tau = k.mu * ((qp[1] - Vs[0]) * tx + (qp[2] - Vs[1]) * ty) / xi;
    if (cq != 0) continue;
    if (surf) {  // Eq. 9 integrand: (p_s - p_inf) / (rho_inf U^2 / 2), tau / (rho_inf U^2 / 2)
      surf[e] = (ps - k.pinf) / 0.5;
      surf[g.nv + e] = tau / 0.5;
    }
    sx += (-(ps - k.pinf) * nx + tau * tx) * L;
    sy += (-(ps - k.pinf) * ny + tau * ty) * L;
  }
  for (int off = 16; off > 0; off >>= 1) {
    sx += __shfl_xor_sync(0xffffffffu, sx, off);
    sy += __shfl_xor_sync(0xffffffffu, sy, off);
  }
  if (threadIdx.x == 0) {
    ds->fpart[2 * blockIdx.x] = sx;
    ds->fpart[2 * blockIdx.x + 1] = sy;
    __threadfence();
    last = atomicAdd(&ds->fdone, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  // the last block: the partials loaded in parallel, then added in block order
  __threadfence();
  for (int b = threadIdx.x; b < (int)gridDim.x; b += FORCE_THREADS) {
    part[2 * b] = *(volatile double *)&ds->fpart[2 * b];
    part[2 * b + 1] = *(volatile double *)&ds->fpart[2 * b + 1];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double fx = 0.0, fy = 0.0;
    for (int b = 0; b < (int)gridDim.x; b++) {
      fx += part[2 * b];
      fy += part[2 * b + 1];
    }
    ds->fdone = 0;
    const double q = 0.5 * k.ref_len;
    ds->force[0] = fx / q;
    ds->force[1] = fy / q;
    ds->force[2] = fx;
    ds->force[3] = fy;
    if (set_accel) {  // Eq. 10: this force sets the body's acceleration for the step
      ds->bF[0] = fx;
      ds->bF[1] = fy;
      ds->bA[0] = fx / k.motion.mass;
      ds->bA[1] = fy / k.motion.mass;
    }
  }
}

void launch_forces_f64(const Consts &k, const Geom &g, const uint8_t *tag, const double *A, bool pert,
                       DevState *ds, cudaStream_t s, bool set_accel, double *surf) {
  const int blocks = std::max(1, std::min(FORCE_BLOCKS, (g.nv + FORCE_SEGS - 1) / FORCE_SEGS));
  k_forces_f64<<<blocks, FORCE_THREADS, 0, s>>>(k, g, tag, A, pert, ds, set_accel, surf);
}

// Sec. 6, Eq. 10: end of a step of a body translating under the fluid force.  The step's constant
// acceleration carries position and velocity over the step (dt of the step; t already advanced).
__global__ void k_body_end(DevState *ds) {
  const double dt = ds->dt;
  for (int d = 0; d < 2; d++) {
    ds->bX[d] = ds->bX[d] + dt * ds->bV[d] + 0.5 * dt * dt * ds->bA[d];
    ds->bV[d] = ds->bV[d] + dt * ds->bA[d];
  }
  ds->bt = ds->t;
}

void launch_body_end(DevState *ds, cudaStream_t s) { k_body_end<<<1, 1, 0, s>>>(ds); }

}  // namespace ibm

using namespace ibm;

// ===========================================================================
// Allocation-free classification + tagging + list compaction.
//
// For callers that cannot allocate device memory themselves or through the
// library: code running where cudaMalloc is unavailable or forbidden (inside
// a host callback, under a memory pool that must not grow, in an embedding
// that owns every device allocation), or a caller that must keep its device
// footprint fixed after start-up.  The caller passes the body and the output
// buffers; the intermediate data (solid flags, per-block counts, bounding box,
// list offsets) lives in the fixed file-scope device array below.  Every GPU
// that loads this library holds that array until the process exits.
// ===========================================================================
namespace {

constexpr int NOALLOC_MAX_CELLS = 1 << 22;  // 4,194,304 cells (e.g. 2048 x 2048)
constexpr int NOALLOC_MAX_VERTS = 4096;
constexpr int NOALLOC_MAX_BLOCKS = (NOALLOC_MAX_CELLS + TAG_BLOCK - 1) / TAG_BLOCK;

struct NoAllocScratch {
  DevState ds;
  double vx[NOALLOC_MAX_VERTS];
  double vy[NOALLOC_MAX_VERTS];
  int blockcounts[4 * NOALLOC_MAX_BLOCKS];
  uint8_t solid[NOALLOC_MAX_CELLS];
};

// total: about 4.3 MiB per device
__device__ __align__(256) NoAllocScratch g_noalloc_scratch;

__global__ void k_noalloc_prepare(const double *__restrict__ verts, int nv, NoAllocScratch *s) {
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    s->vx[v] = verts[2 * v];
    s->vy[v] = verts[2 * v + 1];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double b0 = s->vx[0], b1 = s->vx[0], b2 = s->vy[0], b3 = s->vy[0];
    for (int v = 1; v < nv; v++) {
      if (s->vx[v] < b0) b0 = s->vx[v];
      if (s->vx[v] > b1) b1 = s->vx[v];
      if (s->vy[v] < b2) b2 = s->vy[v];
      if (s->vy[v] > b3) b3 = s->vy[v];
    }
    s->ds.bbox[0] = b0;
    s->ds.bbox[1] = b1;
    s->ds.bbox[2] = b2;
    s->ds.bbox[3] = b3;
    s->ds.err = 0;
  }
}

// same ranking as k_scatter, writing plain cell indices
__global__ void __launch_bounds__(TAG_BLOCK) k_scatter_cells(Consts k, const uint8_t *__restrict__ tag,
                                                             const int *__restrict__ blockoff, const DevState *ds,
                                                             int32_t *__restrict__ cells, int cap) {
  __shared__ int wc[TAG_BLOCK / 32][4];
  const int n = blockIdx.x * TAG_BLOCK + threadIdx.x;
  const int ncell = k.nx * k.ny;
  const int kind = n < ncell ? list_kind(tag[n]) : -1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  int rank = 0;
  for (int q = 0; q < 4; q++) {
    unsigned m = __ballot_sync(0xffffffffu, kind == q);
    if (lane == 0) wc[warp][q] = __popc(m);
    if (kind == q) rank = __popc(m & lt);
  }
  __syncthreads();
  if (kind >= 0) {
    int before = 0;
    for (int w = 0; w < warp; w++) before += wc[w][kind];
    int pos = ds->offset[kind] + blockoff[blockIdx.x * 4 + kind] + before + rank;
    if (pos < cap) cells[pos] = n;
  }
}

std::mutex g_noalloc_mu;
NoAllocScratch *g_noalloc_ptr[256] = {};

}  // namespace

// Defined in the C ABI unit.
extern "C" ibm_status ibm__noalloc_fail(ibm_status s, const char *msg);

extern "C" ibm_status ibm_tag_nodes_noalloc(const ibm_grid *grid, const double *d_verts, int nverts,
                                            uint8_t *d_tags, int32_t *d_cells, int32_t capacity,
                                            int32_t *d_counts, void *cuda_stream) {
  using namespace ibm;
  if (!grid || !d_verts || !d_tags || !d_cells || !d_counts)
    return ibm__noalloc_fail(IBM_EINVAL, "ibm_tag_nodes_noalloc: NULL argument");
  if (grid->nx < 1 || grid->ny < 1 || !(grid->hi[0] > grid->lo[0]) || !(grid->hi[1] > grid->lo[1]))
    return ibm__noalloc_fail(IBM_EINVAL, "ibm_tag_nodes_noalloc: bad grid");
  if ((long long)grid->nx * grid->ny > NOALLOC_MAX_CELLS)
    return ibm__noalloc_fail(IBM_EINVAL, "ibm_tag_nodes_noalloc: grid exceeds the 4194304-cell scratch limit");
  if (nverts < 3 || nverts > NOALLOC_MAX_VERTS)
    return ibm__noalloc_fail(IBM_EINVAL, "ibm_tag_nodes_noalloc: nverts must be in [3, 4096]");
  if (capacity < 0) return ibm__noalloc_fail(IBM_EINVAL, "ibm_tag_nodes_noalloc: negative capacity");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256)
    return ibm__noalloc_fail(IBM_ECUDA, "ibm_tag_nodes_noalloc: no current device");
  NoAllocScratch *s = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void *p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return ibm__noalloc_fail(IBM_ECUDA, "ibm_tag_nodes_noalloc: cudaGetSymbolAddress failed");
      }
      g_noalloc_ptr[dev] = (NoAllocScratch *)p;
    }
    s = g_noalloc_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  Consts k{};
  k.nx = grid->nx;
  k.ny = grid->ny;
  k.x0 = grid->lo[0];
  k.y0 = grid->lo[1];
  k.dx = (grid->hi[0] - grid->lo[0]) / grid->nx;
  k.dy = (grid->hi[1] - grid->lo[1]) / grid->ny;
  Geom g{};
  g.nv = nverts;
  g.vx = s->vx;
  g.vy = s->vy;
  k_noalloc_prepare<<<1, 256, 0, st>>>(d_verts, nverts, s);
  launch_classify(k, g, s->solid, &s->ds, k.nx, k.ny, st);
  const int ncell = k.nx * k.ny;
  const int nblk = (ncell + TAG_BLOCK - 1) / TAG_BLOCK;
  k_tag_count<<<nblk, TAG_BLOCK, 0, st>>>(k, s->solid, d_tags, s->blockcounts);
  k_scan_blocks<<<1, 1024, 0, st>>>(nblk, s->blockcounts, &s->ds, capacity);
  k_scatter_cells<<<nblk, TAG_BLOCK, 0, st>>>(k, d_tags, s->blockcounts, &s->ds, d_cells, capacity);
  cudaError_t e = cudaMemcpyAsync(d_counts, s->ds.count, 4 * sizeof(int32_t), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return ibm__noalloc_fail(IBM_ECUDA, cudaGetErrorString(e));
  return IBM_OK;
}
