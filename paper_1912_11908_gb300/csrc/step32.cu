// Persistent step kernel of the FP32-bulk explicit path: the three SSP-RK3
// stages of one step (Sec. 2) in one launch, per-tile code from stage32.cuh.
//
// Blocks take (stage, tile) items in order from one counter: all items of
// stage 1, then stage 2, then stage 3; within a stage the body tiles first
// (list order), then the other tiles (row-major).  A tile's stage s > 1 reads
// stage s - 1 of its loaded region (three cells around the tile) and, in body
// tiles, of the stencil corners of IB / ghost nodes there, all within two
// tiles of it; the item therefore first waits until every tile within two
// tile columns and rows (wrapping across periodic sides) has published stage
// s - 1.  An item waits only on items handed out before it, which blocks
// already running hold, so the launch always completes; the waits are bounded
// all the same (ERR_TIMEOUT).  Write-after-read is safe by the same order:
// stage 3 of a tile overwrites the mirror of U^n only after its neighbours'
// stage 2, which follows their stage 1, the last reader of it.  Stages
// therefore overlap across the grid instead of each ending with a partly
// filled wave and a launch boundary.
//
// Body tiles lead each stage because their node rebuilds make them the
// longest chains, and the warp schedulers favour a block by its age: blocks
// start claiming in launch order, which hands the first items (stage 1's
// body tiles) to the oldest block on each SM.
#include <cstring>

#include "stage32.cuh"

namespace ibm {

constexpr int STEP_WAIT_SPINS = 1 << 18;

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u32(unsigned int *p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Threads 0..24 each wait for one tile within two tile columns / rows of
// `tile` to reach the completion count `target`; the block then meets at a
// barrier.  A wait that gives up sets ERR_TIMEOUT and the block carries on.
__device__ __forceinline__ void wait_neighbours(const Consts &k, const unsigned int *done, int tile, int ntx, int nty,
                                                unsigned int target, DevState *ds) {
  if (threadIdx.x < 25) {
    int tx = tile % ntx + (int)threadIdx.x % 5 - 2, ty = tile / ntx + (int)threadIdx.x / 5 - 2;
    bool in = true;
    if (tx < 0 || tx >= ntx) {
      if (k.bc[0] == IBM_BC_PERIODIC || k.bc[1] == IBM_BC_PERIODIC) tx = ((tx % ntx) + ntx) % ntx;
      else in = false;
    }
    if (ty < 0 || ty >= nty) {
      if (k.bc[2] == IBM_BC_PERIODIC || k.bc[3] == IBM_BC_PERIODIC) ty = ((ty % nty) + nty) % nty;
      else in = false;
    }
    if (in) {
      const unsigned int *p = done + ty * ntx + tx;
      for (int it = 0; (int)(ld_acquire_u32(p) - target) < 0; it++) {
        // give up after the limit, or at once when another wait of this launch already has
        if (it >= STEP_WAIT_SPINS ||
            ((it & 31) == 31 && (ld_acquire_u32(reinterpret_cast<unsigned int *>(&ds->err)) & ERR_TIMEOUT))) {
          atomicOr(&ds->err, ERR_TIMEOUT);
          break;
        }
        if (it >= 32) __nanosleep(64);
      }
    }
  }
  __syncthreads();
}

// MINB: resident blocks per SM the register allocation must allow (6: 40
// registers, 5: 48 registers).
template <int MINB>
__global__ void __launch_bounds__(256, MINB)
    k_step_f32(Consts k, PertConsts c, float *M, float *F1, float *F2, double *D, const uint8_t *__restrict__ tag,
               const int *__restrict__ sid, const RStencil32 *__restrict__ rs, const uint8_t *__restrict__ tile_body,
               const int *__restrict__ body_tiles, int body_cap, DevState *ds, StepSched *sch, bool fuse_cfl,
               const __grid_constant__ CUtensorMap tm1, const __grid_constant__ CUtensorMap tm2,
               const __grid_constant__ CUtensorMap tm3, int use_tma, int s_first, int s_last) {
  __shared__ TileSmem sm;
  if (threadIdx.x == 0) {  // one barrier for all tensor copies of the block, phases alternating
    tma_init(&sm.mbar);
    sm.mbar_phase = 0u;
  }

  unsigned int *done = reinterpret_cast<unsigned int *>(sch + 1);
  const int ntx = (k.nx + TX - 1) / TX, nty = (k.ny + TY - 1) / TY, nt = ntx * nty;
  // per stage: nb listed body tiles, then every tile in row-major order (listed body tiles skipped); a list
  // that overflowed (an error already flagged) is not used, every tile then comes from the row-major part
  const int nbody = ds->nbody_tiles;
  const int nb = nbody <= body_cap ? nbody : 0;
  const unsigned int per_stage = (unsigned int)(nb + nt), nitems = (unsigned int)(s_last - s_first + 1) * per_stage;
  // completion count of a tile at the start of this launch (written by the previous launch's last block)
  const unsigned int base = 3u * sch->epoch;
  // thread 0 claims an item: per stage, listed body tiles first, then the row-major tiles that are not listed
  auto claim = [&]() -> int {
    for (;;) {
      const unsigned int g = atomicAdd(&sch->next, 1u);
      if (g >= nitems) return -1;
      const unsigned int q = g / per_stage, r = g - q * per_stage;
      const int s = s_first - 1 + (int)q;
      if (r < (unsigned int)nb) return s * nt + body_tiles[r];
      const int tile = (int)(r - nb);
      if (nb == 0 || !tile_body[tile]) return s * nt + tile;  // (stage - 1) * nt + tile
    }
  };
  __shared__ int s_items[2];  // current and next item, alternating
  if (threadIdx.x == 0) s_items[0] = claim();
  __syncthreads();
  for (int it = 0;; it++) {
    const int g = s_items[it & 1];
    if (g < 0) break;
    const int st = g / nt + 1, tile = g - (st - 1) * nt;
    if (st > s_first) wait_neighbours(k, done, tile, ntx, nty, base + st - 1, ds);
    const bool body = tile_body[tile] != 0;
#define IBM_ITEM(S, IN, OUT, TM)                                                                                    \
  do {                                                                                                              \
    if (body)                                                                                                       \
      stage_tile<S, true, false, true, true>(k, c, M, IN, OUT, D, tag, sid, rs, tile_body, nullptr, ds, fuse_cfl,   \
                                             (unsigned int)nt, tile, sm, DualPtrs{}, use_tma ? &TM : nullptr);      \
    else                                                                                                            \
      stage_tile<S, false, false, true, true>(k, c, M, IN, OUT, D, tag, sid, rs, tile_body, nullptr, ds, fuse_cfl,  \
                                              (unsigned int)nt, tile, sm, DualPtrs{}, use_tma ? &TM : nullptr);     \
  } while (0)
    if (st == 1) IBM_ITEM(1, M, F1, tm1);
    else if (st == 2) IBM_ITEM(2, F1, F2, tm2);
    else IBM_ITEM(3, F2, nullptr, tm3);
#undef IBM_ITEM
    // thread 0 (done with its share of the tile) claims the next item; the barrier then both orders every
    // thread's stores before the release of the tile's count and hands the next item to the block
    if (threadIdx.x == 0) s_items[(it + 1) & 1] = claim();
    __syncthreads();
    if (threadIdx.x == 0) st_release_u32(done + tile, base + st);
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&sch->exited, 1u) == gridDim.x - 1) {
      // every block has left the loop: rearm the claim counter and, after stage 3, end the step
      __threadfence();
      if (s_last == 3) {
        const double dt = __ldcg(&ds->dt);
        ds->t = __ldcg(&ds->t) + dt;
        ds->steps = __ldcg(&ds->steps) + 1;
        if (fuse_cfl) {
          ds->dt = __ldcg(&ds->dt_next);
          ds->dtf = __ldcg(&ds->dtf_next);
        }
        sch->epoch = __ldcg(&sch->epoch) + 1u;
      }
      sch->next = 0u;
      sch->exited = 0u;
    }
  }
}

size_t step_sched_bytes(const Consts &k) { return sizeof(StepSched) + sizeof(unsigned int) * (size_t)stage_tiles(k); }

int step_f32_grid(const Consts &k, int variant) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (variant == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_step_f32<5>, 256, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_step_f32<6>, 256, 0);
  long long g = (long long)per * sms;
  const long long items = 3LL * stage_tiles(k);
  if (g > items) g = items;
  return g < 1 ? 1 : (int)g;
}

cudaError_t launch_step_f32(const Consts &k, float *M, float *F1, float *F2, double *D, const uint8_t *tag,
                            const int *sid, const RStencil32 *rs, const uint8_t *tile_body, const int *body_tiles,
                            int body_cap, DevState *ds, StepSched *sch, bool fuse_cfl, const CUtensorMap *tmaps,
                            int variant, int grid, int s_first, int s_last, cudaStream_t s) {
  const PertConsts c = pert_consts(k);
  CUtensorMap tm[3];
  std::memset(tm, 0, sizeof tm);
  const int ut = tmaps ? 1 : 0;
  if (tmaps)
    for (int i = 0; i < 3; i++) tm[i] = tmaps[i];
  // all blocks resident at once
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned int)grid);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (variant == 1)
    return cudaLaunchKernelEx(&cfg, k_step_f32<5>, k, c, M, F1, F2, D, tag, sid, rs, tile_body, body_tiles, body_cap,
                              ds, sch, fuse_cfl, tm[0], tm[1], tm[2], ut, s_first, s_last);
  return cudaLaunchKernelEx(&cfg, k_step_f32<6>, k, c, M, F1, F2, D, tag, sid, rs, tile_body, body_tiles, body_cap,
                            ds, sch, fuse_cfl, tm[0], tm[1], tm[2], ut, s_first, s_last);
}

}  // namespace ibm
