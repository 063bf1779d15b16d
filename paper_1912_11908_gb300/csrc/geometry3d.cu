// 3-D immersed-boundary pre-processing on the GPU (Sec. 3.2, Sec. 4.1-4.2;
// Appendix A's sphere in a cube): ray-casting classification of every node of
// a uniform lattice against a closed triangulated surface, IB / ghost tagging
// over the 6-neighbourhood, ordered node lists, and for every listed node the
// closest surface feature (face, edge or vertex) with its pseudo-normal.
//
// Compiled with -fmad=false: every decision and coordinate comes from IEEE
// basic operations and sqrt evaluated in a fixed order, so tags, lists and
// closest-feature records are reproducible bit for bit.  Face normals and
// the angle-weighted vertex pseudo-normals (Eq. 2, which needs acos) are
// formed once on the host when the body is created.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <utility>
#include <vector>

#include "ibm.h"

extern "C" ibm_status ibm__noalloc_fail(ibm_status s, const char *msg);

namespace {

constexpr int B3 = 256;        // threads per block of the per-node kernels
constexpr int CBLK = 1024;     // nodes per block of the list compaction
constexpr uint8_t T_FLUID = IBM_TAG_FLUID, T_SOLID = IBM_TAG_SOLID, T_IB = IBM_TAG_IB, T_G1 = IBM_TAG_G1;

struct Lattice {
  int nx, ny, nz;
  double lo[3], d[3];
};

struct Mesh {
  int nv, ntri;
  const double *v;    // [nv][3]
  const int *tri;     // [ntri][3]
  const double *fn;   // [ntri][3] unit face normals
  const double *vn;   // [nv][3] unit angle-weighted vertex pseudo-normals
  const int *enb;     // [ntri][3] the face across edge k (vertices k, k+1), -1 if none
  const float4 *fbox; // [ntri][2] per face: box corners (lo, hi), widened by the cull margin (culling only)
  const float4 *fsph; // [ntri] per face: bounding-sphere centre and radius, widened by the cull margin
  double bb[6];       // axis-aligned bounding box: lo x, y, z, hi x, y, z
};

__device__ __forceinline__ void node_xyz(const Lattice &L, long long n, double P[3], int ijk[3]) {
  const long long nxy = (long long)L.nx * L.ny;
  ijk[2] = (int)(n / nxy);
  const long long r = n - (long long)ijk[2] * nxy;
  ijk[1] = (int)(r / L.nx);
  ijk[0] = (int)(r - (long long)ijk[1] * L.nx);
  for (int a = 0; a < 3; a++) P[a] = L.lo[a] + ((double)ijk[a] + 0.5) * L.d[a];
}

// sign of the edge function of edge (a, b) at P in the (u, v) projection, endpoints taken in increasing vertex
// index (the two faces sharing the edge see opposite values), a zero resolved by the symbolic shift of P by
// (eps, eps^2) in (u, v)
__device__ __forceinline__ int edge_sign(const double *pa, int ia, const double *pb, int ib, const double P[3], int u,
                                         int v) {
  int flip = 1;
  if (ib < ia) {
    const double *t = pa;
    pa = pb;
    pb = t;
    flip = -1;
  }
  const double du = pb[u] - pa[u], dv = pb[v] - pa[v];
  const double e = du * (P[v] - pa[v]) - dv * (P[u] - pa[u]);
  int sg = e > 0.0 ? 1 : (e < 0.0 ? -1 : 0);
  if (sg == 0) sg = -dv > 0.0 ? 1 : (-dv < 0.0 ? -1 : 0);
  if (sg == 0) sg = du > 0.0 ? 1 : (du < 0.0 ? -1 : 0);
  return flip * sg;
}

// Sec. 3.2 (Moller-Trumbore, barycentric form): does the ray from P along +axis cross face f ahead of P?
__device__ __forceinline__ int crosses(const Mesh &m, int f, const double P[3], int axis) {
  const int u = axis == 0 ? 1 : (axis == 1 ? 2 : 0), v = axis == 0 ? 2 : (axis == 1 ? 0 : 1);
  const int i0 = __ldg(m.tri + 3 * f), i1 = __ldg(m.tri + 3 * f + 1), i2 = __ldg(m.tri + 3 * f + 2);
  double a[3], b[3], c[3];
  for (int q = 0; q < 3; q++) {
    a[q] = __ldg(m.v + 3 * i0 + q);
    b[q] = __ldg(m.v + 3 * i1 + q);
    c[q] = __ldg(m.v + 3 * i2 + q);
  }
  const int s0 = edge_sign(a, i0, b, i1, P, u, v);
  const int s1 = edge_sign(b, i1, c, i2, P, u, v);
  const int s2 = edge_sign(c, i2, a, i0, P, u, v);
  if (s0 == 0 || s0 != s1 || s1 != s2) return 0;
  const double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
  const double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
  const double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
  if (n[axis] == 0.0) return 0;
  const double num = n[0] * (a[0] - P[0]) + n[1] * (a[1] - P[1]) + n[2] * (a[2] - P[2]);
  return ((num > 0.0 && n[axis] > 0.0) || (num < 0.0 && n[axis] < 0.0)) ? 1 : 0;
}

// classification along lattice lines: one warp per line along `axis`.  Whether the ray from a node crosses a
// face depends on the face's edge functions at the line's two transverse coordinates, the same for every node of
// the line; only "ahead of the node", the sign of n.(a - P), depends on the node.  So the warp collects the faces
// the line crosses once (lanes splitting the faces, the FP32 box cull of the per-node test), then every node of
// the line evaluates its own n.(a - P) over those faces -- the operations of testing every face from every node,
// hence the same parity.  Passes over the three axes accumulate the parities in solid[] (pass 0 writes, pass 1
// adds, pass 2 adds and writes the vote, >= 2 of 3, for nodes inside the surface's bounding box and 0 outside).
// A line crossing more than HCAP faces takes the per-node test over all faces instead.
constexpr int HCAP = 48;

__global__ void __launch_bounds__(B3) k3_classify_lines(Lattice L, Mesh m, int axis, uint8_t *__restrict__ solid) {
  __shared__ double hn[B3 / 32][HCAP][3], ha[B3 / 32][HCAP][3];  // per warp: normal and first vertex of each hit
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int u = axis == 0 ? 1 : (axis == 1 ? 2 : 0), v = axis == 0 ? 2 : (axis == 1 ? 0 : 1);
  const int n[3] = {L.nx, L.ny, L.nz};
  const long long nlines = (long long)n[u] * n[v];
  const long long warps = (long long)gridDim.x * (B3 / 32);
  for (long long li = (long long)blockIdx.x * (B3 / 32) + warp; li < nlines; li += warps) {
    int ijk[3];
    ijk[u] = (int)(li % n[u]);
    ijk[v] = (int)(li / n[u]);
    double P[3];
    P[u] = L.lo[u] + ((double)ijk[u] + 0.5) * L.d[u];
    P[v] = L.lo[v] + ((double)ijk[v] + 0.5) * L.d[v];
    P[axis] = L.lo[axis];
    const bool line_in = !(P[u] < m.bb[u] || P[u] > m.bb[3 + u] || P[v] < m.bb[v] || P[v] > m.bb[3 + v]);
    int cnt = 0;
    if (line_in) {
      const float pu = (float)P[u], pv = (float)P[v];
      for (int f0 = 0; f0 < m.ntri; f0 += 32) {
        const int f = f0 + lane;
        bool hit = false;
        double nf[3] = {0.0, 0.0, 0.0}, af[3] = {0.0, 0.0, 0.0};
        if (f < m.ntri) {
          const float4 lo = __ldg(m.fbox + 2 * f), hi = __ldg(m.fbox + 2 * f + 1);
          const float lu = u == 0 ? lo.x : (u == 1 ? lo.y : lo.z), hu = u == 0 ? hi.x : (u == 1 ? hi.y : hi.z);
          const float lv = v == 0 ? lo.x : (v == 1 ? lo.y : lo.z), hv = v == 0 ? hi.x : (v == 1 ? hi.y : hi.z);
          if (!(pu < lu || pu > hu || pv < lv || pv > hv)) {
            const int i0 = __ldg(m.tri + 3 * f), i1 = __ldg(m.tri + 3 * f + 1), i2 = __ldg(m.tri + 3 * f + 2);
            double A[3], B[3], C[3];
            for (int q = 0; q < 3; q++) {
              A[q] = __ldg(m.v + 3 * i0 + q);
              B[q] = __ldg(m.v + 3 * i1 + q);
              C[q] = __ldg(m.v + 3 * i2 + q);
            }
            const int s0 = edge_sign(A, i0, B, i1, P, u, v);
            const int s1 = edge_sign(B, i1, C, i2, P, u, v);
            const int s2 = edge_sign(C, i2, A, i0, P, u, v);
            if (s0 != 0 && s0 == s1 && s1 == s2) {
              const double e1[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
              const double e2[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
              nf[0] = e1[1] * e2[2] - e1[2] * e2[1];
              nf[1] = e1[2] * e2[0] - e1[0] * e2[2];
              nf[2] = e1[0] * e2[1] - e1[1] * e2[0];
              hit = nf[axis] != 0.0;
              for (int q = 0; q < 3; q++) af[q] = A[q];
            }
          }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, hit);
        if (hit) {
          const int slot = cnt + __popc(bal & ((1u << lane) - 1u));
          if (slot < HCAP)
            for (int q = 0; q < 3; q++) {
              hn[warp][slot][q] = nf[q];
              ha[warp][slot][q] = af[q];
            }
        }
        cnt += __popc(bal);
      }
    }
    __syncwarp();
    if (cnt <= HCAP) {
      for (int t = lane; t < n[axis]; t += 32) {
        ijk[axis] = t;
        double Q[3] = {P[0], P[1], P[2]};
        Q[axis] = L.lo[axis] + ((double)t + 0.5) * L.d[axis];
        int par = 0;
        for (int h = 0; h < cnt; h++) {
          const double num = hn[warp][h][0] * (ha[warp][h][0] - Q[0]) + hn[warp][h][1] * (ha[warp][h][1] - Q[1]) +
                             hn[warp][h][2] * (ha[warp][h][2] - Q[2]);
          const double na = hn[warp][h][axis];
          par += ((num > 0.0 && na > 0.0) || (num < 0.0 && na < 0.0)) ? 1 : 0;
        }
        const long long idx = ((long long)ijk[2] * L.ny + ijk[1]) * L.nx + ijk[0];
        const bool inside = !(Q[0] < m.bb[0] || Q[0] > m.bb[3] || Q[1] < m.bb[1] || Q[1] > m.bb[4] ||
                              Q[2] < m.bb[2] || Q[2] > m.bb[5]);
        const uint8_t p1 = (uint8_t)(par & 1);
        if (axis == 0) solid[idx] = p1;
        else if (axis == 1) solid[idx] = (uint8_t)(solid[idx] + p1);
        else solid[idx] = (uint8_t)(inside && solid[idx] + p1 >= 2);
      }
    } else {
      // more crossings than the warp keeps: every node of the line tests every face (lanes splitting them)
      const float pu = (float)P[u], pv = (float)P[v];
      for (int t = 0; t < n[axis]; t++) {
        ijk[axis] = t;
        double Q[3] = {P[0], P[1], P[2]};
        Q[axis] = L.lo[axis] + ((double)t + 0.5) * L.d[axis];
        const float pa = (float)Q[axis];
        unsigned h = 0;
        for (int f = lane; f < m.ntri; f += 32) {
          const float4 lo = __ldg(m.fbox + 2 * f), hi = __ldg(m.fbox + 2 * f + 1);
          const float lu = u == 0 ? lo.x : (u == 1 ? lo.y : lo.z), hu = u == 0 ? hi.x : (u == 1 ? hi.y : hi.z);
          const float lv = v == 0 ? lo.x : (v == 1 ? lo.y : lo.z), hv = v == 0 ? hi.x : (v == 1 ? hi.y : hi.z);
          const float ha_ = axis == 0 ? hi.x : (axis == 1 ? hi.y : hi.z);
          if (pu < lu || pu > hu || pv < lv || pv > hv || pa > ha_) continue;
          h += (unsigned)crosses(m, f, Q, axis);
        }
        const int par = (int)(__reduce_add_sync(0xffffffffu, h) & 1u);
        if (lane == 0) {
          const long long idx = ((long long)ijk[2] * L.ny + ijk[1]) * L.nx + ijk[0];
          const bool inside = !(Q[0] < m.bb[0] || Q[0] > m.bb[3] || Q[1] < m.bb[1] || Q[1] > m.bb[4] ||
                                Q[2] < m.bb[2] || Q[2] > m.bb[5]);
          if (axis == 0) solid[idx] = (uint8_t)par;
          else if (axis == 1) solid[idx] = (uint8_t)(solid[idx] + par);
          else solid[idx] = (uint8_t)(inside && solid[idx] + par >= 2);
        }
      }
    }
    __syncwarp();  // the hit list is rewritten by the warp's next line
  }
}

__device__ __forceinline__ bool solid_at(const Lattice &L, const uint8_t *__restrict__ solid, int i, int j, int k) {
  return solid[((long long)k * L.ny + j) * L.nx + i] != 0;
}

// Sec. 3.2 / Sec. 5 over the 6-neighbourhood: IB = fluid node with a solid neighbour; G1..G3 = solid node whose
// nearest non-solid node along a lattice line is 1..3 nodes away.  Per block: counts of IB, G1, G2, G3.
__global__ void __launch_bounds__(CBLK) k3_tags(Lattice L, const uint8_t *__restrict__ solid, uint8_t *__restrict__ tags,
                                                int *__restrict__ blockcounts) {
  __shared__ int wc[CBLK / 32][4];
  const long long nn = (long long)L.nx * L.ny * L.nz;
  const long long n = (long long)blockIdx.x * CBLK + threadIdx.x;
  int kind = -1;
  if (n < nn) {
    double P[3];
    int c[3];
    node_xyz(L, n, P, c);
    const int dirs[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
    uint8_t t;
    if (!solid[n]) {
      bool ib = false;
      for (int d = 0; d < 6 && !ib; d++) {
        const int a = c[0] + dirs[d][0], b = c[1] + dirs[d][1], e = c[2] + dirs[d][2];
        if (a >= 0 && a < L.nx && b >= 0 && b < L.ny && e >= 0 && e < L.nz && solid_at(L, solid, a, b, e)) ib = true;
      }
      t = ib ? T_IB : T_FLUID;
    } else {
      t = T_SOLID;
      for (int s = 1; s <= 3 && t == T_SOLID; s++) {
        bool hit = false;
        for (int d = 0; d < 6 && !hit; d++) {
          const int a = c[0] + s * dirs[d][0], b = c[1] + s * dirs[d][1], e = c[2] + s * dirs[d][2];
          if (a >= 0 && a < L.nx && b >= 0 && b < L.ny && e >= 0 && e < L.nz && !solid_at(L, solid, a, b, e))
            hit = true;
        }
        if (hit) t = (uint8_t)(T_G1 + s - 1);
      }
    }
    tags[n] = t;
    kind = t == T_IB ? 0 : (t >= T_G1 ? 1 + t - T_G1 : -1);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = 0; q < 4; q++) {
    const unsigned b = __ballot_sync(0xffffffffu, kind == q);
    if (lane == 0) wc[warp][q] = __popc(b);
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    int s = 0;
    for (int w = 0; w < CBLK / 32; w++) s += wc[w][threadIdx.x];
    blockcounts[4 * blockIdx.x + threadIdx.x] = s;
  }
}

// exclusive offsets of every block within each class's list, and the class totals (counts[0..3]); one block
__global__ void __launch_bounds__(1024) k3_scan(int nblk, int *__restrict__ blockcounts, int *__restrict__ counts) {
  __shared__ int part[1024][4];
  const int per = (nblk + 1023) / 1024, b0 = threadIdx.x * per, b1 = min(nblk, b0 + per);
  int s[4] = {0, 0, 0, 0};
  for (int b = b0; b < b1; b++)
    for (int q = 0; q < 4; q++) s[q] += blockcounts[4 * b + q];
  for (int q = 0; q < 4; q++) part[threadIdx.x][q] = s[q];
  __syncthreads();
  if (threadIdx.x < 4) {  // serial exclusive scan of the 1024 partial sums of one class
    int acc = 0;
    for (int t = 0; t < 1024; t++) {
      const int x = part[t][threadIdx.x];
      part[t][threadIdx.x] = acc;
      acc += x;
    }
    counts[threadIdx.x] = acc;
  }
  __syncthreads();
  int off[4];
  for (int q = 0; q < 4; q++) off[q] = part[threadIdx.x][q];
  for (int b = b0; b < b1; b++)
    for (int q = 0; q < 4; q++) {
      const int x = blockcounts[4 * b + q];
      blockcounts[4 * b + q] = off[q];
      off[q] += x;
    }
}

// listed nodes in row-major order, IB first, then G1, G2, G3; entries past cap are not written
__global__ void __launch_bounds__(CBLK) k3_scatter(Lattice L, const uint8_t *__restrict__ tags,
                                                   const int *__restrict__ blockoff, const int *__restrict__ counts,
                                                   int *__restrict__ nodes, int cap) {
  __shared__ int wc[CBLK / 32][4];
  const long long nn = (long long)L.nx * L.ny * L.nz;
  const long long n = (long long)blockIdx.x * CBLK + threadIdx.x;
  int kind = -1;
  if (n < nn) {
    const uint8_t t = tags[n];
    kind = t == T_IB ? 0 : (t >= T_G1 ? 1 + t - T_G1 : -1);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int rank = 0;
  for (int q = 0; q < 4; q++) {
    const unsigned b = __ballot_sync(0xffffffffu, kind == q);
    if (lane == 0) wc[warp][q] = __popc(b);
    if (kind == q) rank = __popc(b & ((1u << lane) - 1u));
  }
  __syncthreads();
  if (kind >= 0) {
    int pos = blockoff[4 * blockIdx.x + kind] + rank;
    for (int w = 0; w < warp; w++) pos += wc[w][kind];
    for (int q = 0; q < kind; q++) pos += counts[q];
    if (pos < cap) nodes[pos] = (int)n;
  }
}

__device__ __forceinline__ double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// Sec. 4.1: closest point of face f to P -- the plane projection (barycentric normal equations) when it falls
// inside the face, else the nearest point of its three edges (an end vertex when the edge parameter clamps)
__device__ __forceinline__ double face_closest(const Mesh &m, int f, const double P[3], double q[3], int &fk,
                                               int &fe, int &fv) {
  const int t[3] = {__ldg(m.tri + 3 * f), __ldg(m.tri + 3 * f + 1), __ldg(m.tri + 3 * f + 2)};
  double V[3][3];
  for (int k = 0; k < 3; k++)
    for (int d = 0; d < 3; d++) V[k][d] = __ldg(m.v + 3 * t[k] + d);
  const double *A = V[0];
  const double e1[3] = {V[1][0] - A[0], V[1][1] - A[1], V[1][2] - A[2]};
  const double e2[3] = {V[2][0] - A[0], V[2][1] - A[1], V[2][2] - A[2]};
  const double w[3] = {P[0] - A[0], P[1] - A[1], P[2] - A[2]};
  const double a11 = dot3(e1, e1), a12 = dot3(e1, e2), a22 = dot3(e2, e2), b1 = dot3(w, e1), b2 = dot3(w, e2);
  const double det = a11 * a22 - a12 * a12;
  const double s = (b1 * a22 - b2 * a12) / det, r = (a11 * b2 - a12 * b1) / det;
  fk = 0;
  fe = 0;
  fv = 0;
  if (s >= 0.0 && r >= 0.0 && s + r <= 1.0) {
    for (int d = 0; d < 3; d++) q[d] = A[d] + s * e1[d] + r * e2[d];
  } else {
    double dmin = INFINITY;
    for (int k = 0; k < 3; k++) {
      const double *E0 = V[k], *E1 = V[(k + 1) % 3];
      const double ed[3] = {E1[0] - E0[0], E1[1] - E0[1], E1[2] - E0[2]};
      const double pw[3] = {P[0] - E0[0], P[1] - E0[1], P[2] - E0[2]};
      double u = dot3(pw, ed) / dot3(ed, ed);
      int vert = -1;
      if (u <= 0.0) {
        u = 0.0;
        vert = t[k];
      } else if (u >= 1.0) {
        u = 1.0;
        vert = t[(k + 1) % 3];
      }
      const double x[3] = {E0[0] + u * ed[0], E0[1] + u * ed[1], E0[2] + u * ed[2]};
      const double dd[3] = {P[0] - x[0], P[1] - x[1], P[2] - x[2]};
      const double d2 = dot3(dd, dd);
      if (d2 < dmin) {
        dmin = d2;
        q[0] = x[0];
        q[1] = x[1];
        q[2] = x[2];
        fk = vert >= 0 ? IBM_FEATURE_VERTEX : IBM_FEATURE_EDGE;
        fe = k;
        fv = vert;
      }
    }
  }
  const double dq[3] = {P[0] - q[0], P[1] - q[1], P[2] - q[2]};
  return dot3(dq, dq);
}

// Sec. 4.1-4.2: closest feature of every listed node (one warp per node, lanes splitting the faces, the
// lowest face index among equal distances) and its pseudo-normal: the face normal, the angle-weighted vertex
// normal (Eq. 2) or the normalised sum of the two faces' normals at an edge (Eq. 3)
__global__ void __launch_bounds__(B3) k3_closest(Lattice L, Mesh m, const int *__restrict__ nodes,
                                                 const int *__restrict__ counts, int cap,
                                                 ibm_closest3d *__restrict__ rec) {
  const int total = min(cap, counts[0] + counts[1] + counts[2] + counts[3]);
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (B3 / 32);
  for (int e = blockIdx.x * (B3 / 32) + (threadIdx.x >> 5); e < total; e += warps) {
    const long long n = nodes[e];
    double P[3];
    int ijk[3];
    node_xyz(L, n, P, ijk);
    // bounding spheres (FP32, widened by the cull margin): the nearest possible and the farthest possible
    // distance of every face; a face whose nearest possible distance exceeds the smallest farthest possible
    // distance of any face cannot hold the closest point (the margin is far above FP32 rounding, and a face
    // within it is tested exactly)
    const float pf[3] = {(float)P[0], (float)P[1], (float)P[2]};
    float ub = INFINITY;
    for (int f = lane; f < m.ntri; f += 32) {
      const float4 s = __ldg(m.fsph + f);
      const float dx = pf[0] - s.x, dy = pf[1] - s.y, dz = pf[2] - s.z;
      ub = fminf(ub, sqrtf(dx * dx + dy * dy + dz * dz) + s.w);
    }
    for (int off = 16; off > 0; off >>= 1) ub = fminf(ub, __shfl_xor_sync(0xffffffffu, ub, off));
    double best = INFINITY, bq[3] = {0.0, 0.0, 0.0};
    int bf = -1, bk = 0, be = 0, bv = 0;
    for (int f = lane; f < m.ntri; f += 32) {
      const float4 s = __ldg(m.fsph + f);
      const float dx = pf[0] - s.x, dy = pf[1] - s.y, dz = pf[2] - s.z;
      if (sqrtf(dx * dx + dy * dy + dz * dz) - s.w > ub) continue;
      double q[3];
      int fk, fe, fv;
      const double d2 = face_closest(m, f, P, q, fk, fe, fv);
      if (d2 < best) {  // ascending f within the lane: the first minimum is kept
        best = d2;
        bf = f;
        bk = fk;
        be = fe;
        bv = fv;
        bq[0] = q[0];
        bq[1] = q[1];
        bq[2] = q[2];
      }
    }
    // lexicographic (distance, face) minimum over the warp
    double md = best;
    int mf = bf < 0 ? 0x7fffffff : bf;
    for (int off = 16; off > 0; off >>= 1) {
      const double od = __shfl_xor_sync(0xffffffffu, md, off);
      const int of = __shfl_xor_sync(0xffffffffu, mf, off);
      if (od < md || (od == md && of < mf)) {
        md = od;
        mf = of;
      }
    }
    if (bf == mf) {  // the lane that holds the winning face writes the record
      double nn[3];
      if (bk == IBM_FEATURE_FACE) {
        for (int d = 0; d < 3; d++) nn[d] = m.fn[3 * bf + d];
      } else if (bk == IBM_FEATURE_VERTEX) {
        for (int d = 0; d < 3; d++) nn[d] = m.vn[3 * bv + d];
      } else {
        const int g = m.enb[3 * bf + be];
        for (int d = 0; d < 3; d++) nn[d] = m.fn[3 * bf + d] + (g >= 0 ? m.fn[3 * g + d] : 0.0);
        const double Ln = sqrt(dot3(nn, nn));
        if (Ln > 0.0)
          for (int d = 0; d < 3; d++) nn[d] = nn[d] / Ln;
      }
      ibm_closest3d o;
      o.node = (int32_t)n;
      o.tri = bf;
      o.kind = bk;
      o.reserved = 0;
      for (int d = 0; d < 3; d++) {
        o.cp[d] = bq[d];
        o.n[d] = nn[d];
      }
      rec[e] = o;
    }
  }
}

// host: unit face normals and angle-weighted vertex pseudo-normals (Eq. 2), in the order of the faces
void host_normals(int nv, const double *v, int ntri, const int *tri, std::vector<double> &fn, std::vector<double> &vn) {
  fn.assign((size_t)3 * ntri, 0.0);
  vn.assign((size_t)3 * nv, 0.0);
  auto dot = [](const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; };
  auto unit = [&](double *a) {
    const double Ln = std::sqrt(dot(a, a));
    if (Ln > 0.0) {
      a[0] = a[0] / Ln;
      a[1] = a[1] / Ln;
      a[2] = a[2] / Ln;
    }
  };
  for (int f = 0; f < ntri; f++) {
    const int *t = tri + 3 * f;
    const double *A = v + 3 * t[0], *B = v + 3 * t[1], *C = v + 3 * t[2];
    const double e1[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
    const double e2[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
    double *n = &fn[(size_t)3 * f];
    n[0] = e1[1] * e2[2] - e1[2] * e2[1];
    n[1] = e1[2] * e2[0] - e1[0] * e2[2];
    n[2] = e1[0] * e2[1] - e1[1] * e2[0];
    unit(n);
    for (int k = 0; k < 3; k++) {
      const double *O = v + 3 * t[k], *X = v + 3 * t[(k + 1) % 3], *Y = v + 3 * t[(k + 2) % 3];
      const double a[3] = {X[0] - O[0], X[1] - O[1], X[2] - O[2]};
      const double b[3] = {Y[0] - O[0], Y[1] - O[1], Y[2] - O[2]};
      const double cosv = dot(a, b) / std::sqrt(dot(a, a) * dot(b, b));
      const double ang = std::acos(std::fmax(-1.0, std::fmin(1.0, cosv)));  // interior angle at vertex t[k]
      for (int d = 0; d < 3; d++) vn[(size_t)3 * t[k] + d] += ang * n[d];
    }
  }
  for (int k = 0; k < nv; k++) unit(&vn[(size_t)3 * k]);
}

// Sec. 4.3-4.6 and Sec. 5 in 3-D: the interpolation cube around X over the cell centres and its weights --
// trilinear when all eight corners carry an allowed tag, otherwise 1 / r^2 over the allowed ones (a corner hit
// exactly takes all the weight); returns the corner mask
__device__ int cube_weights(const Lattice &L, const uint8_t *__restrict__ tags, const double X[3], unsigned allowed,
                            int o[3], double w[8]) {
  const int n[3] = {L.nx, L.ny, L.nz};
  for (int a = 0; a < 3; a++) o[a] = (int)floor((X[a] - L.lo[a]) / L.d[a] - 0.5);
  int mask = 0;
  for (int b = 0; b < 8; b++) {
    const int ci = o[0] + (b & 1), cj = o[1] + (b >> 1 & 1), ck = o[2] + (b >> 2);
    w[b] = 0.0;
    if (ci < 0 || ci >= n[0] || cj < 0 || cj >= n[1] || ck < 0 || ck >= n[2]) continue;
    if (allowed & (1u << tags[((long long)ck * n[1] + cj) * n[0] + ci])) mask |= 1 << b;
  }
  if (mask == 255) {
    double f[3];
    for (int a = 0; a < 3; a++) {
      const double c0 = L.lo[a] + ((double)o[a] + 0.5) * L.d[a];
      f[a] = (X[a] - c0) / L.d[a];
    }
    for (int b = 0; b < 8; b++) {
      const double wx = (b & 1) ? f[0] : 1.0 - f[0];
      const double wy = (b >> 1 & 1) ? f[1] : 1.0 - f[1];
      const double wz = (b >> 2) ? f[2] : 1.0 - f[2];
      w[b] = wx * wy * wz;
    }
  } else if (mask != 0) {
    double inv[8];
    int hit = -1;
    for (int b = 0; b < 8; b++) inv[b] = 0.0;
    for (int b = 0; b < 8 && hit < 0; b++) {
      if (!(mask >> b & 1)) continue;
      const int idx[3] = {o[0] + (b & 1), o[1] + (b >> 1 & 1), o[2] + (b >> 2)};
      double r2 = 0.0;
      for (int a = 0; a < 3; a++) {
        const double r = X[a] - (L.lo[a] + ((double)idx[a] + 0.5) * L.d[a]);
        r2 = r2 + r * r;
      }
      if (r2 == 0.0) hit = b;
      else inv[b] = 1.0 / r2;
    }
    if (hit >= 0) {
      w[hit] = 1.0;
    } else {
      double sum = 0.0;
      for (int b = 0; b < 8; b++)
        if (mask >> b & 1) sum += inv[b];
      for (int b = 0; b < 8; b++)
        if (mask >> b & 1) w[b] = inv[b] / sum;
    }
  }
  return mask;
}

// one stencil per listed node (IB first, then G1..G3, as listed): boundary point P' = X - xi_node n on the
// tangent plane through the closest point, probe one cell diagonal h beyond an IB node, mirror image point of a
// ghost node (at least dmin / 2 from P'), pushed out by dmin up to three times while the cube has no valid
// corner; a node left without one counts in *nerr
__global__ void __launch_bounds__(B3) k3_stencils(Lattice L, const uint8_t *__restrict__ tags,
                                                  const int *__restrict__ nodes, const int *__restrict__ counts,
                                                  int cap, const ibm_closest3d *__restrict__ rec, double h,
                                                  double dmin, ibm_stencil3d *__restrict__ out,
                                                  int *__restrict__ nerr) {
  const int c0 = counts[0], c1 = counts[1], c2 = counts[2];
  const int total = min(cap, c0 + c1 + c2 + counts[3]);
  const int e = blockIdx.x * B3 + threadIdx.x;
  if (e >= total) return;
  const int kind = e < c0 ? 0 : e < c0 + c1 ? 1 : e < c0 + c1 + c2 ? 2 : 3;
  const ibm_closest3d r = rec[e];
  double X[3];
  int ijk[3];
  node_xyz(L, nodes[e], X, ijk);
  const double xi_node = (X[0] - r.cp[0]) * r.n[0] + (X[1] - r.cp[1]) * r.n[1] + (X[2] - r.cp[2]) * r.n[2];
  double b[3];
  for (int a = 0; a < 3; a++) b[a] = X[a] - xi_node * r.n[a];
  double xi_probe;
  if (kind == 0) {
    xi_probe = xi_node + h;
  } else {
    xi_probe = -xi_node;
    if (xi_probe < 0.5 * dmin) xi_probe = 0.5 * dmin;
  }
  const unsigned allowed = kind == 0 ? (1u << T_FLUID) : ((1u << T_FLUID) | (1u << T_IB));
  ibm_stencil3d s;
  int o[3] = {0, 0, 0}, mask = 0, nstep = 0;
  for (;;) {
    double P[3];
    for (int a = 0; a < 3; a++) P[a] = b[a] + xi_probe * r.n[a];
    mask = cube_weights(L, tags, P, allowed, o, s.w);
    if (mask != 0 || nstep == 3) break;
    xi_probe = xi_probe + dmin;
    nstep++;
  }
  if (mask == 0) atomicAdd(nerr, 1);
  s.node = nodes[e];
  s.kind = kind;
  s.region = r.kind;
  s.nstep = nstep;
  s.i0 = o[0];
  s.j0 = o[1];
  s.k0 = o[2];
  s.mask = mask;
  for (int a = 0; a < 3; a++) {
    s.n[a] = r.n[a];
    s.b[a] = b[a];
  }
  s.xi_node = xi_node;
  s.xi_probe = xi_probe;
  out[e] = s;
}

// Sec. 6 (Eq. 9) in 3-D: the probe of each triangle one cell diagonal out along its normal from its centroid
// (mn: per triangle the centroid and the unit normal, 6 doubles), pushed out by dmin up to three times while its
// cube has no fluid corner; the record's b is the centroid, xi_probe the probe distance, node the triangle
__global__ void __launch_bounds__(B3) k3_surface_stencils(Lattice L, const uint8_t *__restrict__ tags,
                                                          const double *__restrict__ mn, int ntri, double h,
                                                          double dmin, ibm_stencil3d *__restrict__ out) {
  const int f = blockIdx.x * B3 + threadIdx.x;
  if (f >= ntri) return;
  const double m[3] = {mn[6 * f], mn[6 * f + 1], mn[6 * f + 2]}, n[3] = {mn[6 * f + 3], mn[6 * f + 4], mn[6 * f + 5]};
  ibm_stencil3d s;
  double xi = h;
  int o[3] = {0, 0, 0}, mask = 0, nstep = 0;
  for (int st = 0; st <= 3; st++) {
    const double P[3] = {m[0] + xi * n[0], m[1] + xi * n[1], m[2] + xi * n[2]};
    mask = cube_weights(L, tags, P, 1u << T_FLUID, o, s.w);
    if (mask) break;
    if (st < 3) {
      xi = xi + dmin;
      nstep++;
    }
  }
  s.node = f;
  s.kind = 0;
  s.region = IBM_FEATURE_FACE;
  s.nstep = nstep;
  s.i0 = o[0];
  s.j0 = o[1];
  s.k0 = o[2];
  s.mask = mask;
  for (int a = 0; a < 3; a++) {
    s.n[a] = n[a];
    s.b[a] = m[a];
  }
  s.xi_node = 0.0;
  s.xi_probe = xi;
  out[f] = s;
}

}  // namespace

struct ibm_body3d {
  Mesh m{};
  char *mem = nullptr;       // mesh data on the device
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  Lattice L{};
  long long nn = 0;          // lattice nodes of the last classification
  int nblk = 0, cap = 0;
  uint8_t *solid = nullptr, *tags = nullptr;
  int *blockcounts = nullptr, *counts = nullptr, *nodes = nullptr;
  ibm_closest3d *rec = nullptr;
  bool classified = false;
};

static ibm_status cuda_fail(cudaError_t e) { return ibm__noalloc_fail(IBM_ECUDA, cudaGetErrorString(e)); }

static void free_lattice(ibm_body3d *b) {
  cudaFree(b->solid);
  cudaFree(b->tags);
  cudaFree(b->blockcounts);
  cudaFree(b->counts);
  cudaFree(b->nodes);
  cudaFree(b->rec);
  b->solid = b->tags = nullptr;
  b->blockcounts = b->counts = b->nodes = nullptr;
  b->rec = nullptr;
  b->nn = 0;
}

extern "C" ibm_status ibm_body3d_create(const double *verts, int nverts, const int32_t *tris, int ntris,
                                        void *cuda_stream, ibm_body3d **out) {
  if (!out || !verts || !tris || nverts < 4 || ntris < 4) return ibm__noalloc_fail(IBM_EINVAL, "ibm_body3d_create: bad mesh");
  *out = nullptr;
  for (int k = 0; k < 3 * ntris; k++)
    if (tris[k] < 0 || tris[k] >= nverts) return ibm__noalloc_fail(IBM_EINVAL, "ibm_body3d_create: vertex index out of range");
  std::vector<double> fn, vn;
  host_normals(nverts, verts, ntris, tris, fn, vn);
  // the face across each edge: the first face (in index order) holding the reversed directed edge
  std::map<std::pair<int, int>, int> first;
  for (int f = 0; f < ntris; f++)
    for (int k = 0; k < 3; k++) first.emplace(std::make_pair(tris[3 * f + k], tris[3 * f + (k + 1) % 3]), f);
  std::vector<int> enb((size_t)3 * ntris, -1);
  for (int f = 0; f < ntris; f++)
    for (int k = 0; k < 3; k++) {
      auto it = first.find(std::make_pair(tris[3 * f + (k + 1) % 3], tris[3 * f + k]));
      if (it != first.end()) enb[(size_t)3 * f + k] = it->second;
    }
  // per-face boxes and bounding spheres for the FP32 culls, widened by a margin of 1e-5 of the mesh extent
  double ext = 0.0;
  {
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int k = 0; k < nverts; k++)
      for (int a = 0; a < 3; a++) {
        lo[a] = std::min(lo[a], verts[3 * k + a]);
        hi[a] = std::max(hi[a], verts[3 * k + a]);
      }
    for (int a = 0; a < 3; a++) ext = std::max(ext, std::max(std::fabs(lo[a]), std::fabs(hi[a])));
    ext = std::max(ext, 1.0);
  }
  const double margin = 1e-5 * ext;
  std::vector<float4> fbox((size_t)2 * ntris), fsph((size_t)ntris);
  for (int f = 0; f < ntris; f++) {
    const double *V[3] = {verts + 3 * tris[3 * f], verts + 3 * tris[3 * f + 1], verts + 3 * tris[3 * f + 2]};
    double lo[3], hi[3], cen[3], r2 = 0.0;
    for (int a = 0; a < 3; a++) {
      lo[a] = std::min(V[0][a], std::min(V[1][a], V[2][a])) - margin;
      hi[a] = std::max(V[0][a], std::max(V[1][a], V[2][a])) + margin;
      cen[a] = (V[0][a] + V[1][a] + V[2][a]) / 3.0;
    }
    for (int k = 0; k < 3; k++) {
      const double dx = V[k][0] - cen[0], dy = V[k][1] - cen[1], dz = V[k][2] - cen[2];
      r2 = std::max(r2, dx * dx + dy * dy + dz * dz);
    }
    fbox[(size_t)2 * f] = make_float4((float)lo[0], (float)lo[1], (float)lo[2], 0.f);
    fbox[(size_t)2 * f + 1] = make_float4((float)hi[0], (float)hi[1], (float)hi[2], 0.f);
    fsph[f] = make_float4((float)cen[0], (float)cen[1], (float)cen[2], (float)(std::sqrt(r2) + margin));
  }
  ibm_body3d *b = new ibm_body3d();
  b->m.nv = nverts;
  b->m.ntri = ntris;
  for (int a = 0; a < 3; a++) {
    b->m.bb[a] = INFINITY;
    b->m.bb[3 + a] = -INFINITY;
  }
  for (int k = 0; k < nverts; k++)
    for (int a = 0; a < 3; a++) {
      b->m.bb[a] = std::min(b->m.bb[a], verts[3 * k + a]);
      b->m.bb[3 + a] = std::max(b->m.bb[3 + a], verts[3 * k + a]);
    }
  const size_t sv = (size_t)3 * nverts * sizeof(double), st = (size_t)3 * ntris * sizeof(int),
               sf = (size_t)3 * ntris * sizeof(double);
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t sbx = (size_t)2 * ntris * sizeof(float4), ssp = (size_t)ntris * sizeof(float4);
  const size_t total = up(sv) * 2 + up(st) * 2 + up(sf) + up(sbx) + up(ssp);
  cudaError_t e = cudaMalloc(&b->mem, total);
  if (e != cudaSuccess) {
    delete b;
    return ibm__noalloc_fail(IBM_ENOMEM, "ibm_body3d_create: device allocation failed");
  }
  char *p = b->mem;
  double *dv = (double *)p;
  p += up(sv);
  double *dvn = (double *)p;
  p += up(sv);
  int *dt = (int *)p;
  p += up(st);
  int *den = (int *)p;
  p += up(st);
  double *dfn = (double *)p;
  p += up(sf);
  float4 *dbx = (float4 *)p;
  p += up(sbx);
  float4 *dsp = (float4 *)p;
  if (cuda_stream) {
    b->stream = (cudaStream_t)cuda_stream;
  } else {
    e = cudaStreamCreate(&b->stream);
    b->own_stream = e == cudaSuccess;
  }
  if (e == cudaSuccess) e = cudaMemcpy(dv, verts, sv, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dvn, vn.data(), sv, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dt, tris, st, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(den, enb.data(), st, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dfn, fn.data(), sf, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dbx, fbox.data(), sbx, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dsp, fsph.data(), ssp, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    ibm_body3d_destroy(b);
    return cuda_fail(e);
  }
  b->m.v = dv;
  b->m.vn = dvn;
  b->m.tri = dt;
  b->m.enb = den;
  b->m.fn = dfn;
  b->m.fbox = dbx;
  b->m.fsph = dsp;
  *out = b;
  return IBM_OK;
}

extern "C" ibm_status ibm_body3d_classify(ibm_body3d *b, const ibm_grid3d *g) {
  if (!b || !g || g->nx < 1 || g->ny < 1 || g->nz < 1) return ibm__noalloc_fail(IBM_EINVAL, "ibm_body3d_classify: bad grid");
  const long long nn = (long long)g->nx * g->ny * g->nz;
  if (nn > (1LL << 31) - 1) return ibm__noalloc_fail(IBM_EINVAL, "ibm_body3d_classify: more than 2^31 - 1 nodes");
  for (int a = 0; a < 3; a++)
    if (!(g->hi[a] > g->lo[a])) return ibm__noalloc_fail(IBM_EINVAL, "ibm_body3d_classify: empty domain");
  Lattice L;
  L.nx = g->nx;
  L.ny = g->ny;
  L.nz = g->nz;
  const int nd[3] = {g->nx, g->ny, g->nz};
  for (int a = 0; a < 3; a++) {
    L.lo[a] = g->lo[a];
    L.d[a] = (g->hi[a] - g->lo[a]) / (double)nd[a];
  }
  // listed nodes lie within three nodes of the bounding box
  long long cap = 1;
  for (int a = 0; a < 3; a++) {
    long long i0 = (long long)std::floor((b->m.bb[a] - L.lo[a]) / L.d[a] - 0.5) - 4;
    long long i1 = (long long)std::ceil((b->m.bb[3 + a] - L.lo[a]) / L.d[a] - 0.5) + 4;
    i0 = std::max(0LL, i0);
    i1 = std::min((long long)nd[a] - 1, i1);
    cap *= std::max(0LL, i1 - i0 + 1);
  }
  cap = std::max(1LL, std::min(cap, nn));
  cudaError_t e = cudaSuccess;
  if (nn != b->nn || (int)cap != b->cap) {
    e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return cuda_fail(e);
    free_lattice(b);
    b->nblk = (int)((nn + CBLK - 1) / CBLK);
    if (e == cudaSuccess) e = cudaMalloc(&b->solid, (size_t)nn);
    if (e == cudaSuccess) e = cudaMalloc(&b->tags, (size_t)nn);
    if (e == cudaSuccess) e = cudaMalloc(&b->blockcounts, (size_t)4 * b->nblk * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->counts, 4 * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->nodes, (size_t)cap * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->rec, (size_t)cap * sizeof(ibm_closest3d));
    if (e != cudaSuccess) {
      free_lattice(b);
      return ibm__noalloc_fail(IBM_ENOMEM, "ibm_body3d_classify: device allocation failed");
    }
    b->nn = nn;
    b->cap = (int)cap;
  }
  b->L = L;
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int gw = nsm * 8;  // 8 blocks of 8 warps per SM, striding over the lines (classification) or nodes
  for (int axis = 0; axis < 3; axis++) k3_classify_lines<<<gw, B3, 0, b->stream>>>(L, b->m, axis, b->solid);
  k3_tags<<<b->nblk, CBLK, 0, b->stream>>>(L, b->solid, b->tags, b->blockcounts);
  k3_scan<<<1, 1024, 0, b->stream>>>(b->nblk, b->blockcounts, b->counts);
  k3_scatter<<<b->nblk, CBLK, 0, b->stream>>>(L, b->tags, b->blockcounts, b->counts, b->nodes, b->cap);
  k3_closest<<<gw, B3, 0, b->stream>>>(L, b->m, b->nodes, b->counts, b->cap, b->rec);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e);
  b->classified = true;
  return IBM_OK;
}

extern "C" ibm_status ibm_body3d_get(ibm_body3d *b, int what, void *dst, size_t bytes) {
  if (!b || !dst) return ibm__noalloc_fail(IBM_EINVAL, "ibm_body3d_get: NULL argument");
  if (!b->classified) return ibm__noalloc_fail(IBM_ESTATE, "ibm_body3d_get: not classified");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  int cnt[4];
  e = cudaMemcpy(cnt, b->counts, sizeof(cnt), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e);
  const long long total = (long long)cnt[0] + cnt[1] + cnt[2] + cnt[3];
  const int n = (int)std::min<long long>(total, b->cap);
  switch (what) {
    case IBM_3D_TAGS:
      if (bytes < (size_t)b->nn) return ibm__noalloc_fail(IBM_EINVAL, "ibm_body3d_get: dst too small");
      e = cudaMemcpy(dst, b->tags, (size_t)b->nn, cudaMemcpyDeviceToHost);
      break;
    case IBM_3D_COUNTS:
      if (bytes < sizeof(cnt)) return ibm__noalloc_fail(IBM_EINVAL, "ibm_body3d_get: dst too small");
      std::memcpy(dst, cnt, sizeof(cnt));
      break;
    case IBM_3D_NODES:
      if (bytes < (size_t)n * sizeof(int32_t)) return ibm__noalloc_fail(IBM_EINVAL, "ibm_body3d_get: dst too small");
      if (n) e = cudaMemcpy(dst, b->nodes, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost);
      break;
    case IBM_3D_CLOSEST:
      if (bytes < (size_t)n * sizeof(ibm_closest3d)) return ibm__noalloc_fail(IBM_EINVAL, "ibm_body3d_get: dst too small");
      if (n) e = cudaMemcpy(dst, b->rec, (size_t)n * sizeof(ibm_closest3d), cudaMemcpyDeviceToHost);
      break;
    default:
      return ibm__noalloc_fail(IBM_EINVAL, "ibm_body3d_get: unknown quantity");
  }
  if (e != cudaSuccess) return cuda_fail(e);
  if (total > b->cap) return ibm__noalloc_fail(IBM_ECAPACITY, "ibm_body3d_get: more listed nodes than the capacity");
  return IBM_OK;
}

extern "C" ibm_status ibm_body3d_destroy(ibm_body3d *b) {
  if (!b) return IBM_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  free_lattice(b);
  cudaFree(b->mem);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
  return IBM_OK;
}

// The 3-D flow solver's view of a classification: enqueue the stencils of the listed nodes (k3_stencils) on the
// body's stream, with h the probe distance and dmin the push-out step, into out (capacity b->cap entries);
// *nerr (device) receives the number of nodes without a valid corner.  Returns the device tags and per-class
// counts and the list capacity.
ibm_status ibm__body3d_stencils(ibm_body3d *b, double h, double dmin, ibm_stencil3d *out, int *nerr,
                                const uint8_t **tags, const int **counts, int *cap) {
  if (!b || !b->classified) return ibm__noalloc_fail(IBM_ESTATE, "3-D stencils: body not classified");
  k3_stencils<<<(b->cap + B3 - 1) / B3, B3, 0, b->stream>>>(b->L, b->tags, b->nodes, b->counts, b->cap, b->rec, h,
                                                           dmin, out, nerr);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e);
  *tags = b->tags;
  *counts = b->counts;
  *cap = b->cap;
  return IBM_OK;
}

int ibm__body3d_capacity(const ibm_body3d *b) { return b ? b->cap : 0; }

// The force probes of the 3-D flow solver (k3_surface_stencils) on the body's stream.
ibm_status ibm__surface3d_stencils(ibm_body3d *b, const double *mn, int ntri, double h, double dmin,
                                   ibm_stencil3d *out) {
  if (!b || !b->classified) return ibm__noalloc_fail(IBM_ESTATE, "3-D surface probes: body not classified");
  if (ntri > 0)
    k3_surface_stencils<<<(ntri + B3 - 1) / B3, B3, 0, b->stream>>>(b->L, b->tags, mn, ntri, h, dmin, out);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? IBM_OK : cuda_fail(e);
}
