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
#include <mutex>

#include "ibm_internal.cuh"

namespace ibm {

// ---------------------------------------------------------------------------
// Sec. 4.2: pseudo-normals.  Segment k of the CCW polyline runs from vertex k
// to k+1; its outward normal is the travel direction turned clockwise.  The
// 2-D vertex pseudo-normal weights its two incident segments equally (each
// incident "face" enters Eq. 2 / Eq. 3 with the same weight) and is
// normalised.  One thread per vertex.
// ---------------------------------------------------------------------------
__global__ void k_normals(int nv, const double *__restrict__ v, double *snx, double *sny, double *vnx,
                          double *vny) {
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
}

void launch_normals(int nv, const double *v, double *snx, double *sny, double *vnx, double *vny,
                    cudaStream_t s) {
  if (nv <= 0) return;
  k_normals<<<(nv + 127) / 128, 128, 0, s>>>(nv, v, snx, sny, vnx, vny);
}

// ---------------------------------------------------------------------------
// Body pose at the start of the step (prescribed translation) and its
// axis-aligned bounding box.  One block.
// ---------------------------------------------------------------------------
__global__ void k_pose(Consts k, Geom g, DevState *ds) {
  __shared__ double X[2];
  if (threadIdx.x == 0) {
    double V[2], A[2], P[2];
    motion_at(k.motion, ds->t, P, V, A);
    X[0] = P[0];
    X[1] = P[1];
    ds->pos[0] = P[0];
    ds->pos[1] = P[1];
  }
  __syncthreads();
  for (int v = threadIdx.x; v < g.nv; v += blockDim.x) {
    g.vx[v] = g.vref[2 * v] + X[0];
    g.vy[v] = g.vref[2 * v + 1] + X[1];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double b0 = g.vx[0], b1 = g.vx[0], b2 = g.vy[0], b3 = g.vy[0];
    for (int v = 1; v < g.nv; v++) {
      if (g.vx[v] < b0) b0 = g.vx[v];
      if (g.vx[v] > b1) b1 = g.vx[v];
      if (g.vy[v] < b2) b2 = g.vy[v];
      if (g.vy[v] > b3) b3 = g.vy[v];
    }
    ds->bbox[0] = b0;
    ds->bbox[1] = b1;
    ds->bbox[2] = b2;
    ds->bbox[3] = b3;
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
  __shared__ int part[1024][4];
  __shared__ int tot[4];
  const int tid = threadIdx.x;
  const int per = (nblk + 1023) / 1024;
  const int b0 = tid * per, b1 = min(nblk, b0 + per);
  int s[4] = {0, 0, 0, 0};
  for (int b = b0; b < b1; b++)
    for (int q = 0; q < 4; q++) s[q] += blockcounts[b * 4 + q];
  for (int q = 0; q < 4; q++) part[tid][q] = s[q];
  __syncthreads();
  // Hillis-Steele inclusive scan over the 1024 partial sums
  for (int off = 1; off < 1024; off <<= 1) {
    int v[4];
    for (int q = 0; q < 4; q++) v[q] = tid >= off ? part[tid - off][q] : 0;
    __syncthreads();
    for (int q = 0; q < 4; q++) part[tid][q] += v[q];
    __syncthreads();
  }
  if (tid == 1023)
    for (int q = 0; q < 4; q++) tot[q] = part[1023][q];
  __syncthreads();
  int run[4];
  for (int q = 0; q < 4; q++) run[q] = part[tid][q] - s[q];
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

// lexicographic (value, index) minimum across a warp; every lane gets the winner's lane
__device__ __forceinline__ int warp_argmin(double v, int idx) {
  int src = threadIdx.x & 31;
  for (int off = 16; off > 0; off >>= 1) {
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

// Sec. 4.1-4.6, Sec. 5: one stencil per listed node, one warp per node.  The
// lanes split the segments of the two exhaustive searches (closest feature,
// boundary point); the warp keeps the (distance, segment) lexicographic
// minimum, which is the first minimum of a sequential scan.
__global__ void __launch_bounds__(128) k_stencils(Consts k, Geom g, const uint8_t *__restrict__ tag,
                                                  ibm_stencil *__restrict__ st, int cap, DevState *ds) {
  const int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int total = min(ds->offset[4], cap);
  if (e >= total) return;
  ibm_stencil s = st[e];
  const int kind = s.kind;
  const int i = s.cell % k.nx, j = s.cell / k.nx;
  const double px = k.x0 + ((double)i + 0.5) * k.dx;
  const double py = k.y0 + ((double)j + 0.5) * k.dy;
  const int nv = g.nv;
  // closest feature (Sec. 4.1)
  double best = INFINITY, bcx = 0.0, bcy = 0.0;
  int bseg = 0x7fffffff, bfeat = 0, breg = 0;
  for (int kk = lane; kk < nv; kk += 32) {
    const int k1 = (kk + 1 == nv) ? 0 : kk + 1;
    const double ax = g.vx[kk], ay = g.vy[kk], bx = g.vx[k1], by = g.vy[k1];
    const double ex = bx - ax, ey = by - ay;
    const double wx = px - ax, wy = py - ay;
    const double num = wx * ex + wy * ey;
    const double den = ex * ex + ey * ey;
    double cx, cy;
    int f, r;
    if (num <= 0.0) {
      cx = ax; cy = ay; f = kk; r = IBM_REGION_VERTEX;
    } else if (num >= den) {
      cx = bx; cy = by; f = k1; r = IBM_REGION_VERTEX;
    } else {
      const double t = num / den;
      cx = ax + t * ex; cy = ay + t * ey; f = kk; r = IBM_REGION_FACE;
    }
    const double ddx = px - cx, ddy = py - cy;
    const double d2 = ddx * ddx + ddy * ddy;
    if (d2 < best) {
      best = d2; bseg = kk; bfeat = f; breg = r; bcx = cx; bcy = cy;
    }
  }
  int src = warp_argmin(best, bseg);
  const int feat = __shfl_sync(0xffffffffu, bfeat, src);
  const int region = __shfl_sync(0xffffffffu, breg, src);
  const double ccx = __shfl_sync(0xffffffffu, bcx, src);
  const double ccy = __shfl_sync(0xffffffffu, bcy, src);
  double nx, ny;
  if (region == IBM_REGION_FACE) {
    nx = g.snx[feat];
    ny = g.sny[feat];
  } else {
    nx = g.vnx[feat];
    ny = g.vny[feat];
  }
  // boundary point on the line along the local normal (Sec. 4.3)
  const bool ghost = kind > 0;
  double bs_best = INFINITY, bs_s = 0.0;
  int bs_seg = 0x7fffffff;
  for (int kk = lane; kk < nv; kk += 32) {
    const int k1 = (kk + 1 == nv) ? 0 : kk + 1;
    const double ax = g.vx[kk], ay = g.vy[kk];
    const double ex = g.vx[k1] - ax, ey = g.vy[k1] - ay;
    const double den = ex * ny - ey * nx;
    if (den == 0.0) continue;
    const double wx = px - ax, wy = py - ay;
    const double u = (wx * ny - wy * nx) / den;
    if (u < 0.0 || u > 1.0) continue;
    const double sv = (wx * ey - wy * ex) / den;
    if (ghost ? (sv < 0.0) : (sv > 0.0)) continue;
    const double as = fabs(sv);
    if (as < bs_best) {
      bs_best = as; bs_s = sv; bs_seg = kk;
    }
  }
  src = warp_argmin(bs_best, bs_seg);
  const double found_abs = __shfl_sync(0xffffffffu, bs_best, src);
  const double bsv = __shfl_sync(0xffffffffu, bs_s, src);
  if (lane != 0) return;
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
  st[e] = s;
}

void launch_stencils(const Consts &k, const Geom &g, const uint8_t *tag, ibm_stencil *st, int cap, DevState *ds,
                     cudaStream_t s) {
  if (cap <= 0) return;
  k_stencils<<<(unsigned)(((long long)cap * 32 + 127) / 128), 128, 0, s>>>(k, g, tag, st, cap, ds);
}

// ---------------------------------------------------------------------------
// Sec. 6, Eq. 9: force on the body, midpoint rule per segment; surface
// pressure and wall shear from a probe one diagonal spacing out along the
// segment normal (inverse-distance weighted, Sec. 4.6); free-stream pressure
// subtracted.  One block; fixed-order tree reduction (deterministic).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_forces_f64(Consts k, Geom g, const uint8_t *__restrict__ tag,
                                                    const double *__restrict__ A, bool pert, DevState *ds) {
  __shared__ double rx[256], ry[256];
  double V[2], Acc[2], X[2];
  motion_at(k.motion, ds->t, X, V, Acc);
  double sx = 0.0, sy = 0.0;
  for (int e = threadIdx.x; e < g.nv; e += blockDim.x) {
    int e1 = (e + 1 == g.nv) ? 0 : e + 1;
    double ax = g.vx[e], ay = g.vy[e];
    double ex = g.vx[e1] - ax, ey = g.vy[e1] - ay;
    double L = sqrt(ex * ex + ey * ey);
    double tx = ex / L, ty = ey / L;
    double nx = ty, ny = -tx;
    double mx = ax + 0.5 * ex, my = ay + 0.5 * ey;
    double xi = k.h, w[4];
    int i0 = 0, j0 = 0, mask = 0;
    for (int stp = 0; stp <= 3; stp++) {
      mask = interp_square(k, tag, mx + xi * nx, my + xi * ny, ALLOW_FLUID, &i0, &j0, w);
      if (mask) break;
      if (stp < 3) xi = xi + k.dmin;
    }
    if (!mask) continue;
    double qp[4] = {0.0, 0.0, 0.0, 0.0};
    for (int q = 0; q < 4; q++) {
      if (!(mask >> q & 1)) continue;
      long long id = cidx(k, i0 + (q & 1), j0 + (q >> 1));
      double U0 = A[id], U1 = A[id + k.plane], U2 = A[id + 2 * k.plane], U3 = A[id + 3 * k.plane];
      if (pert) {  // perturbation state dU -> absolute conserved
        U3 = k.Uinf[3] + U3 + k.Hinf * U0;
        U0 = 1.0 + U0;
        U1 = k.Uinf[1] + U1;
        U2 = k.Uinf[2] + U2;
      }
      double r = U0, u = U1 / r, v = U2 / r;
      double pr = (k.gamma - 1.0) * (U3 - 0.5 * r * (u * u + v * v));
      double T = pr / (r * k.R);
      qp[0] += w[q] * pr;
      qp[1] += w[q] * u;
      qp[2] += w[q] * v;
      qp[3] += w[q] * T;
    }
    double rho_p = qp[0] / (k.R * qp[3]);
    double gn = -rho_p * (nx * Acc[0] + ny * Acc[1]);
    double ps = qp[0] - xi * gn;
    double tau = k.mu * ((qp[1] - V[0]) * tx + (qp[2] - V[1]) * ty) / xi;
    sx += (-(ps - k.pinf) * nx + tau * tx) * L;
    sy += (-(ps - k.pinf) * ny + tau * ty) * L;
  }
  rx[threadIdx.x] = sx;
  ry[threadIdx.x] = sy;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if (threadIdx.x < off) {
      rx[threadIdx.x] += rx[threadIdx.x + off];
      ry[threadIdx.x] += ry[threadIdx.x + off];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double q = 0.5 * k.ref_len;
    ds->force[0] = rx[0] / q;
    ds->force[1] = ry[0] / q;
    ds->force[2] = rx[0];
    ds->force[3] = ry[0];
  }
}

void launch_forces_f64(const Consts &k, const Geom &g, const uint8_t *tag, const double *A, bool pert,
                       DevState *ds, cudaStream_t s) {
  k_forces_f64<<<1, 256, 0, s>>>(k, g, tag, A, pert, ds);
}

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
