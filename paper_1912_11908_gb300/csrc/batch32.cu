// Block-table stage kernels of the request loop: one launch per RK stage over
// all member cases of a group (the dual-time pseudo-stage form is in
// dual32.cu, beside the single-case dual-time launch that shares it).  Kept in a module of their own: linked into the
// single-case module, these kernels slowed the replay of single-case step
// graphs by ~10% on GB300 (measured; kernel durations themselves unchanged).
#include "stage32.cuh"

namespace ibm {

// All entries of a stage in one launch: the body-tile entries of every member
// first (they carry the node rebuilds), then the plain-tile entries; blocks
// walk the combined table with a grid stride, so a grid smaller than the
// table makes the launch persistent.  Per entry the block runs the per-tile
// code of the case the entry falls in (the same source as the single-case
// kernels; compiled separately, so FP32 roundings may differ between them).
// Launched with programmatic dependent launch, its blocks are resident while
// the previous stage's last blocks finish (they wait at the top for it to
// complete).
// TVD / QUAD: the TVD-2 reconstruction and / or the quadratic IB / ghost reconstruction compiled in (a group
// holds cases of one variant)
template <int STAGE, bool TVD, bool QUAD>
__global__ void __launch_bounds__(256, 6) k_stage_f32_batch_one(const __grid_constant__ StageBatch b) {
  __shared__ TileSmem sm;
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int nbody = b.body_start[b.n], total = nbody + b.plain_start[b.n];
  for (int e = blockIdx.x; e < total; e += gridDim.x) {
    const bool body = e < nbody;
    const int *start = body ? b.body_start : b.plain_start;
    const int ee = body ? e : e - nbody;
    int q = 0;
    while (q + 1 < b.n && start[q + 1] <= ee) q++;
    const StageCase &sc = b.cs[q];
    const float *In = STAGE == 1 ? sc.M : (STAGE == 2 ? sc.F1 : sc.F2);
    float *Out = STAGE == 1 ? sc.F1 : (STAGE == 2 ? sc.F2 : nullptr);
    if (body)
      stage_tile<STAGE, true, false, false, false, TVD, QUAD>(sc.k, sc.c, sc.M, In, Out, sc.D, sc.tag, sc.sid, sc.rs,
                                                              sc.tile_body, sc.body_tiles, sc.ds, sc.fuse_cfl != 0,
                                                              sc.ncfl, ee - start[q], sm, DualPtrs{}, nullptr,
                                                              sc.rsq);
    else
      stage_tile<STAGE, false, false, false, false, TVD, QUAD>(sc.k, sc.c, sc.M, In, Out, sc.D, sc.tag, sc.sid,
                                                               sc.rs, sc.tile_body, sc.body_tiles, sc.ds,
                                                               sc.fuse_cfl != 0, sc.ncfl, ee - start[q], sm,
                                                               DualPtrs{}, nullptr, sc.rsq);
    __syncthreads();  // shared memory is reused by the next entry
  }
}

cudaError_t launch_stage_f32_batch_one(const StageBatch &b, int stage, int grid, bool pdl, cudaStream_t s) {
  const int total = b.body_start[b.n] + b.plain_start[b.n];
  if (total == 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned int)(grid > 0 && grid < total ? grid : total));
  cfg.blockDim = dim3(256);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  const bool tvd = b.cs[0].k.tvd2 != 0, quad = b.cs[0].k.quad != 0;
  if (quad)
    for (int q = 0; q < b.n; q++)
      if (!b.cs[q].rsq) return cudaErrorInvalidValue;  // the quadratic kernels read the second probes
#define IBM_BATCH(S, T, Q) cudaLaunchKernelEx(&cfg, k_stage_f32_batch_one<S, T, Q>, b)
#define IBM_BATCH_S(S)                                                                                          \
  (tvd ? (quad ? IBM_BATCH(S, true, true) : IBM_BATCH(S, true, false))                                          \
       : (quad ? IBM_BATCH(S, false, true) : IBM_BATCH(S, false, false)))
  const cudaError_t e = stage == 1 ? IBM_BATCH_S(1) : stage == 2 ? IBM_BATCH_S(2) : IBM_BATCH_S(3);
#undef IBM_BATCH_S
#undef IBM_BATCH
  return e;
}

void build_stage_batch(const StageCase *cases, int n, StageBatch *b) {
  b->n = n;
  b->plain_start[0] = b->body_start[0] = 0;
  for (int q = 0; q < n; q++) {
    b->cs[q] = cases[q];
    b->plain_start[q + 1] = b->plain_start[q] + cases[q].nt;
    b->body_start[q + 1] = b->body_start[q] + cases[q].nb;
  }
}

void fill_stage_case(const Consts &k, float *M, float *F1, float *F2, double *D, const uint8_t *tag, const int *sid,
                     const RStencil32 *rs, const uint8_t *tile_body, const int *body_tiles, int body_cap,
                     DevState *ds, bool fuse_cfl, StageCase *out) {
  out->k = k;
  out->c = pert_consts(k);
  out->M = M;
  out->F1 = F1;
  out->F2 = F2;
  out->D = D;
  out->tag = tag;
  out->sid = sid;
  out->rs = rs;
  out->tile_body = tile_body;
  out->body_tiles = body_tiles;
  out->ds = ds;
  out->nt = stage_tiles(k);
  out->nb = body_cap > 0 ? body_cap : 0;
  out->fuse_cfl = fuse_cfl ? 1 : 0;
  out->ncfl = (unsigned int)(out->nt + out->nb);
  out->B = out->C = out->Q0 = nullptr;
  out->G = nullptr;
  out->rsq = nullptr;
}


}  // namespace ibm
