// FP32-bulk flow kernels of one case: the FP64 master's perturbation form back
// to absolute variables, the CFL reduction, compact stencils, body-tile lists
// and the stage kernels (per-tile code in stage32.cuh).  (A state written by
// the caller takes k_set_state of flow.cu.)
#include <algorithm>
#include <cstring>
#include <mutex>

#include "stage32.cuh"

namespace ibm {

// FP64 perturbation -> FP64 absolute conserved
__global__ void k_pert_to_abs64(Consts k, const double *__restrict__ D, double *__restrict__ A) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= k.plane) return;
  const long long P = k.plane;
  const double d = D[n];
  A[n] = 1.0 + d;
  A[n + P] = k.Uinf[1] + D[n + P];
  A[n + 2 * P] = k.Uinf[2] + D[n + 2 * P];
  A[n + 3 * P] = k.Uinf[3] + D[n + 3 * P] + k.Hinf * d;
}

void launch_pert_to_abs64(const Consts &k, const double *D, double *A, cudaStream_t s) {
  k_pert_to_abs64<<<(unsigned)((k.plane + 255) / 256), 256, 0, s>>>(k, D, A);
}

// CFL rule (same expression as the FP64 path) evaluated in FP32 on the mirror
// of U^n; the last block converts the maximum into dt.
__global__ void __launch_bounds__(256) k_dt_f32(Consts k, PertConsts c, const float *__restrict__ M,
                                                const uint8_t *__restrict__ tag, DevState *ds) {
  // a warp on 32 cells of a row, the block's eight warps on eight rows, striding down the grid; the state is
  // loaded whatever the tag and the loop unrolled, so that the loads of several rows leave together (few blocks:
  // each block's maximum and completion are atomics on one address)
  const int i = blockIdx.x * 32 + (threadIdx.x & 31);
  const long long P = k.plane;
  const float idx = c.idx, idy = c.idy;
  const float vis = (float)((2.0 * k.gamma * k.mu / k.prandtl) * (1.0 / (k.dx * k.dx) + 1.0 / (k.dy * k.dy)));
  float lmax = 0.f;
  if (i < k.nx) {
#pragma unroll 4
    for (int j = blockIdx.y * 8 + (threadIdx.x >> 5); j < k.ny; j += gridDim.y * 8) {
      const long long id = cidx(k, i, j);
      const float dr = M[id], mx = M[id + P], my = M[id + 2 * P], w = M[id + 3 * P];
      if (tag[j * k.nx + i] == FLUID || (k.ib_advance && tag[j * k.nx + i] == IB)) {
        float u, v, pp, Tp;
        pert_prim(c, dr, mx, my, w, u, v, pp, Tp);
        const float r = 1.f + dr;
        const float cs = sqrtf(c.gamma * (c.R + pp) / r);
        lmax = fmaxf(lmax, (fabsf(u) + cs) * idx + (fabsf(v) + cs) * idy + vis / r);
      }
    }
  }
  for (int off = 16; off > 0; off >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, off));
  __shared__ float wm[8];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = lmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = wm[0];
    for (int w = 1; w < 8; w++) m = fmaxf(m, wm[w]);
    atomicMax(&ds->lmax_bits, (unsigned long long)__double_as_longlong((double)m));
    finish_cfl(k, ds, gridDim.x * gridDim.y);
  }
}

void launch_dt_f32(const Consts &k, const float *M, const uint8_t *tag, DevState *ds, cudaStream_t s,
                   int *nlaunch) {
  if (k.dt_fixed > 0.0) return;
  // about two blocks per SM
  const int gx = (k.nx + 31) / 32, rows8 = (k.ny + 7) / 8;
  const int gy = std::max(1, std::min(rows8, (2 * 152 + gx - 1) / gx));
  k_dt_f32<<<dim3((unsigned)gx, (unsigned)gy), 256, 0, s>>>(k, pert_consts(k), M, tag, ds);
  *nlaunch += 1;
}

// FP32 copy of every IB / ghost stencil and the cell -> stencil map used by the
// fused reconstruction (sid must be -1 on entry)
__global__ void k_compact_stencils(Consts k, const ibm_stencil *__restrict__ st, RStencil32 *__restrict__ rs,
                                   RStencilQ *__restrict__ rsq, int *__restrict__ sid, int cap,
                                   const DevState *__restrict__ ds) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= min(ds->offset[4], cap)) return;
  const ibm_stencil s = st[e];
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
  const bool pitching = k.motion.kind == IBM_MOTION_PITCH;
  r.rx = pitching ? (float)(s.bx - k.motion.pivot[0]) : 0.f;
  r.ry = pitching ? (float)(s.by - k.motion.pivot[1]) : 0.f;
  rs[e] = r;
  sid[s.cell] = e;
  if (rsq) rsq[e] = quad_stencil(k, s);
}

void launch_compact_stencils(const Consts &k, const ibm_stencil *st, RStencil32 *rs, RStencilQ *rsq, int *sid,
                             int cap, const DevState *ds, cudaStream_t s) {
  cudaMemsetAsync(sid, 0xff, sizeof(int) * (size_t)k.nx * k.ny, s);
  if (cap <= 0) return;
  k_compact_stencils<<<(cap + 127) / 128, 128, 0, s>>>(k, st, rs, rsq, sid, cap, ds);
}

// A case stepped on its own: one block per tile (plain) or body-tile slot.
// MINB: resident blocks per SM the register allocation must allow (0: left to
// the compiler, 40 registers; 5: 48 registers; 4: about 60 registers) -- the
// autotuner picks one per grid size.
template <int STAGE, bool BODY, int MINB>
__global__ void __launch_bounds__(256, MINB) k_stage_f32(Consts k, PertConsts c, float *Mn, const float *__restrict__ In,
                                                   float *Out, double *D, const uint8_t *__restrict__ tag,
                                                   const int *__restrict__ sid, const RStencil32 *__restrict__ rs,
                                                   const uint8_t *__restrict__ tile_body,
                                                   const int *__restrict__ body_tiles, DevState *ds, bool fuse_cfl,
                                                   unsigned int ncfl, const __grid_constant__ CUtensorMap tmap,
                                                   int use_tma) {
  __shared__ TileSmem sm;
  stage_tile<STAGE, BODY, false, true>(k, c, Mn, In, Out, D, tag, sid, rs, tile_body, body_tiles, ds, fuse_cfl, ncfl,
                                       (int)blockIdx.x, sm, DualPtrs{}, use_tma ? &tmap : nullptr);
}

// All tiles of a stage in one launch: blocks [0, nb) are body-tile slots
// (dispatched first: they carry the node rebuilds, the longest chains), the
// rest one block per tile (tiles in the body list return at once).  With
// programmatic dependent launch the next stage's launch may begin once every
// block of this one has started; its blocks then wait at the top for this
// grid to complete and its stores to become visible, so the next stage's
// blocks are resident when the tail of this one ends.
template <int STAGE, int MINB>
__global__ void __launch_bounds__(256, MINB)
    k_stage_f32_one(Consts k, PertConsts c, float *Mn, const float *__restrict__ In, float *Out, double *D,
                    const uint8_t *__restrict__ tag, const int *__restrict__ sid, const RStencil32 *__restrict__ rs,
                    const uint8_t *__restrict__ tile_body, const int *__restrict__ body_tiles, int nb, DevState *ds,
                    bool fuse_cfl, unsigned int ncfl, const __grid_constant__ CUtensorMap tmap, int use_tma) {
  __shared__ TileSmem sm;
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int b = (int)blockIdx.x;
  if (b < nb)
    stage_tile<STAGE, true, false, true>(k, c, Mn, In, Out, D, tag, sid, rs, tile_body, body_tiles, ds, fuse_cfl,
                                         ncfl, b, sm, DualPtrs{}, use_tma ? &tmap : nullptr);
  else
    stage_tile<STAGE, false, false, true>(k, c, Mn, In, Out, D, tag, sid, rs, tile_body, body_tiles, ds, fuse_cfl,
                                          ncfl, b - nb, sm, DualPtrs{}, use_tma ? &tmap : nullptr);
}

// The same stage with the TVD-2 reconstruction (Sec. 2) and / or the quadratic IB / ghost reconstruction
// (Sec. 4.5, Sec. 5) compiled in: a case with either takes this kernel in every launch form (the two-stream
// form runs it as one launch on the case stream), so that the default kernels carry neither.
template <int STAGE, bool TVD, bool QUAD>
__global__ void __launch_bounds__(256, 6)
    k_stage_f32_var(Consts k, PertConsts c, float *Mn, const float *__restrict__ In, float *Out, double *D,
                    const uint8_t *__restrict__ tag, const int *__restrict__ sid, const RStencil32 *__restrict__ rs,
                    const uint8_t *__restrict__ tile_body, const int *__restrict__ body_tiles, int nb, DevState *ds,
                    bool fuse_cfl, unsigned int ncfl, const __grid_constant__ CUtensorMap tmap, int use_tma,
                    const RStencilQ *__restrict__ rsq) {
  __shared__ TileSmem sm;
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int b = (int)blockIdx.x;
  if (b < nb)
    stage_tile<STAGE, true, false, true, false, TVD, QUAD>(k, c, Mn, In, Out, D, tag, sid, rs, tile_body, body_tiles,
                                                           ds, fuse_cfl, ncfl, b, sm, DualPtrs{},
                                                           use_tma ? &tmap : nullptr, rsq);
  else
    stage_tile<STAGE, false, false, true, false, TVD, QUAD>(k, c, Mn, In, Out, D, tag, sid, rs, tile_body,
                                                            body_tiles, ds, fuse_cfl, ncfl, b - nb, sm, DualPtrs{},
                                                            use_tma ? &tmap : nullptr, rsq);
}

int stage_tiles(const Consts &k) { return ((k.nx + TX - 1) / TX) * ((k.ny + TY - 1) / TY); }

// does the tile's loaded range [lo, hi] (before domain mapping) along one axis
// reach the cells [blo, bhi]?  Outflow and free-stream sides map into / drop
// the outside cells, so clamping is exact-or-conservative; a periodic side
// that the range crosses wraps it, so that case answers yes
__device__ __forceinline__ bool axis_reaches(int lo, int hi, int n, int bc_lo, int bc_hi, int blo, int bhi) {
  if ((lo < 0 && bc_lo == IBM_BC_PERIODIC) || (hi >= n && bc_hi == IBM_BC_PERIODIC)) return true;
  lo = max(lo, 0);
  hi = min(hi, n - 1);
  return lo <= bhi && hi >= blo;
}

// flag every stage tile whose cells or 3-cell halo (after domain mapping) hold
// an IB or ghost node; one warp per tile.  Non-fluid tags lie within one cell
// of the cells whose centres fall in the body's bounding box, so a tile whose
// loaded region misses that cell range (ds->bcell, 3-cell margin) has none.
__global__ void k_tile_flags(Consts k, const uint8_t *__restrict__ tag, uint8_t *__restrict__ tile_body,
                             const DevState *__restrict__ ds, int has_body) {
  const int ntx = (k.nx + TX - 1) / TX, nt = ntx * ((k.ny + TY - 1) / TY);
  const int tile = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (tile >= nt) return;
  const int i0 = (tile % ntx) * TX, j0 = (tile / ntx) * TY;
  if (!has_body) {
    if (lane == 0) tile_body[tile] = 0;
    return;
  }
  const int ilo = ds->bcell[0], ihi = ds->bcell[1], jlo = ds->bcell[2], jhi = ds->bcell[3];
  if (!axis_reaches(i0 - NG, i0 + TX + NG - 1, k.nx, k.bc[0], k.bc[1], ilo, ihi) ||
      !axis_reaches(j0 - NG, j0 + TY + NG - 1, k.ny, k.bc[2], k.bc[3], jlo, jhi)) {
    if (lane == 0) tile_body[tile] = 0;
    return;
  }
  bool hit = false;
  for (int m = lane; m < HX * HY; m += 32) {
    int gi = i0 - NG + m % HX, gj = j0 - NG + m / HX;
    if (!halo_map(k, gi, gj)) continue;
    const uint8_t t = tag[gj * k.nx + gi];
    hit |= (t == IB || t >= G1);
  }
  hit = __any_sync(0xffffffffu, hit);
  if (lane == 0) tile_body[tile] = hit ? 1 : 0;
}

// compact the flagged tiles (ascending) into body_tiles; one block
__global__ void __launch_bounds__(1024) k_tile_list(int nt, const uint8_t *__restrict__ tile_body,
                                                    int *__restrict__ body_tiles, int body_cap, DevState *ds) {
  __shared__ int part[1024];
  const int per = (nt + 1023) / 1024;
  const int t0 = threadIdx.x * per, t1 = min(nt, t0 + per);
  int cnt = 0;
  for (int t = t0; t < t1; t++) cnt += tile_body[t];
  part[threadIdx.x] = cnt;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const int v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int pos = part[threadIdx.x] - cnt;
  for (int t = t0; t < t1; t++)
    if (tile_body[t]) {
      if (pos < body_cap) body_tiles[pos] = t;
      pos++;
    }
  if (threadIdx.x == 1023) {
    ds->nbody_tiles = min(part[1023], body_cap);
    if (part[1023] > body_cap) ds->err |= ERR_CAPACITY;
  }
}

void launch_tile_lists(const Consts &k, const uint8_t *tag, uint8_t *tile_body, int *body_tiles, int body_cap,
                       DevState *ds, bool has_body, cudaStream_t s) {
  const int nt = stage_tiles(k);
  k_tile_flags<<<(nt + 7) / 8, 256, 0, s>>>(k, tag, tile_body, ds, has_body ? 1 : 0);
  k_tile_list<<<1, 1024, 0, s>>>(nt, tile_body, body_tiles, body_cap, ds);
}

void launch_stage_f32(const Consts &k, int stage, float *Mn, const float *In, float *Out, double *D,
                      const uint8_t *tag, const int *sid, const RStencil32 *rs, const uint8_t *tile_body,
                      const int *body_tiles, int body_cap, DevState *ds, bool fuse_cfl, cudaStream_t s,
                      cudaStream_t sb, int plain_variant, bool with_body, const CUtensorMap *tmap,
                      const RStencilQ *rsq) {
  if (k.tvd2 || k.quad) {  // the variant kernel holds plain and body tiles: one launch on the case stream
    launch_stage_f32_one(k, stage, Mn, In, Out, D, tag, sid, rs, tile_body, body_tiles, with_body ? body_cap : 0, ds,
                         fuse_cfl, plain_variant, tmap, false, s, rsq);
    return;
  }
  PertConsts c = pert_consts(k);
  const int nt = stage_tiles(k);
  const int nb = body_cap > 0 ? body_cap : 0;
  const unsigned int ncfl = (unsigned int)(nt + nb);
  CUtensorMap tm;
  std::memset(&tm, 0, sizeof tm);
  if (tmap) tm = *tmap;
  const int ut = tmap ? 1 : 0;
#define IBM_ARGS k, c, Mn, In, Out, D, tag, sid, rs, tile_body, body_tiles, ds, fuse_cfl, ncfl, tm, ut
#define IBM_STAGE_PAIR(S)                                                      \
  do {                                                                         \
    if (nb && with_body) k_stage_f32<S, true, 0><<<nb, 256, 0, sb>>>(IBM_ARGS); \
    if (plain_variant == 1)                                                    \
      k_stage_f32<S, false, 5><<<nt, 256, 0, s>>>(IBM_ARGS);                   \
    else if (plain_variant == 2)                                               \
      k_stage_f32<S, false, 4><<<nt, 256, 0, s>>>(IBM_ARGS);                   \
    else                                                                       \
      k_stage_f32<S, false, 0><<<nt, 256, 0, s>>>(IBM_ARGS);                   \
  } while (0)
  if (stage == 1) IBM_STAGE_PAIR(1);
  else if (stage == 2) IBM_STAGE_PAIR(2);
  else IBM_STAGE_PAIR(3);
#undef IBM_STAGE_PAIR
#undef IBM_ARGS
}

cudaError_t launch_stage_f32_one(const Consts &k, int stage, float *Mn, const float *In, float *Out, double *D,
                                 const uint8_t *tag, const int *sid, const RStencil32 *rs, const uint8_t *tile_body,
                                 const int *body_tiles, int body_cap, DevState *ds, bool fuse_cfl, int plain_variant,
                                 const CUtensorMap *tmap, bool pdl, cudaStream_t s, const RStencilQ *rsq) {
  if (k.quad && !rsq) return cudaErrorInvalidValue;  // the quadratic kernels read the second probes
  const PertConsts c = pert_consts(k);
  const int nt = stage_tiles(k);
  const int nb = body_cap > 0 ? body_cap : 0;
  const unsigned int ncfl = (unsigned int)(nt + nb);
  CUtensorMap tm;
  std::memset(&tm, 0, sizeof tm);
  if (tmap) tm = *tmap;
  const int ut = tmap ? 1 : 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned int)(nt + nb));
  cfg.blockDim = dim3(256);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
#define IBM_ONE(S, MB)                                                                                        \
  cudaLaunchKernelEx(&cfg, k_stage_f32_one<S, MB>, k, c, Mn, In, Out, D, tag, sid, rs, tile_body, body_tiles, nb, \
                     ds, fuse_cfl, ncfl, tm, ut)
#define IBM_ONE_V(S) (plain_variant == 1 ? IBM_ONE(S, 5) : plain_variant == 2 ? IBM_ONE(S, 4) : IBM_ONE(S, 6))
#define IBM_VAR(S, T, Q)                                                                                       \
  cudaLaunchKernelEx(&cfg, k_stage_f32_var<S, T, Q>, k, c, Mn, In, Out, D, tag, sid, rs, tile_body, body_tiles, nb, \
                     ds, fuse_cfl, ncfl, tm, ut, rsq)
#define IBM_VAR_S(S) \
  (k.tvd2 && k.quad ? IBM_VAR(S, true, true) : k.tvd2 ? IBM_VAR(S, true, false) : IBM_VAR(S, false, true))
  cudaError_t e = k.tvd2 || k.quad ? (stage == 1 ? IBM_VAR_S(1) : stage == 2 ? IBM_VAR_S(2) : IBM_VAR_S(3))
                                   : (stage == 1 ? IBM_ONE_V(1) : stage == 2 ? IBM_ONE_V(2) : IBM_ONE_V(3));
#undef IBM_VAR_S
#undef IBM_VAR
#undef IBM_ONE_V
#undef IBM_ONE
  return e;
}

// Tensor maps of the three FP32 stage inputs (mirror of U^n, U^(1), U^(2)) for
// the TMA tile staging: 3-D tensors (pitch, rows, 4 planes) of floats, box
// TMA_W x HY x 4.  The encoder is the driver's cuTensorMapEncodeTiled, looked
// up through the runtime (no link-time dependence on the driver library).
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

bool make_stage_tmaps(const Consts &k, float *const arrays[3], CUtensorMap out[3]) {
  static std::once_flag once;
  static EncodeTiledFn encode = nullptr;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      encode = (EncodeTiledFn)p;
    cudaGetLastError();
  });
  if (!encode || k.pitch < TMA_W || k.rows < HY) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)k.pitch, (cuuint64_t)k.rows, 4};
  const cuuint64_t strides[2] = {(cuuint64_t)k.pitch * sizeof(float), (cuuint64_t)k.plane * sizeof(float)};
  const cuuint32_t box[3] = {(cuuint32_t)TMA_W, (cuuint32_t)HY, 4};
  const cuuint32_t estr[3] = {1, 1, 1};
  for (int q = 0; q < 3; q++) {
    if (encode(&out[q], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, arrays[q], dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  return true;
}

}  // namespace ibm
