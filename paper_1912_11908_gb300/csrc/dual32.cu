// Dual-time pseudo stages in FP32-bulk form (Sec. 2): FP32 perturbation
// residual with preconditioned faces, FP64 point-implicit update (per-tile
// code in stage32.cuh).  A module of its own, like the block-table kernels:
// the explicit stage kernels' module holds only what an explicit step
// launches.
#include "stage32.cuh"

namespace ibm {

// Dual-time pseudo stage of one case (FP32 residual, FP64 point-implicit
// update): plain tiles and body tiles as for the explicit stages.
template <int STAGE, bool BODY>
__global__ void __launch_bounds__(256) k_dual_f32(Consts k, PertConsts c, const float *__restrict__ In,
                                                  float *Out32, double *D, const uint8_t *__restrict__ tag,
                                                  const int *__restrict__ sid, const RStencil32 *__restrict__ rs,
                                                  const uint8_t *__restrict__ tile_body,
                                                  const int *__restrict__ body_tiles, DevState *ds, unsigned int ncfl,
                                                  DualPtrs dp) {
  __shared__ TileSmem sm;
  stage_tile<STAGE, BODY, true>(k, c, nullptr, In, Out32, D, tag, sid, rs, tile_body, body_tiles, ds, false, ncfl,
                                (int)blockIdx.x, sm, dp);
}

// The same pseudo stage as one launch: body-tile slots [0, nb) first, then one
// block per tile; with programmatic dependent launch its blocks are resident
// while the previous pseudo stage's last blocks finish (they wait at the top
// for it to complete).
template <int STAGE>
__global__ void __launch_bounds__(256) k_dual_f32_one(Consts k, PertConsts c, const float *__restrict__ In,
                                                      float *Out32, double *D, const uint8_t *__restrict__ tag,
                                                      const int *__restrict__ sid,
                                                      const RStencil32 *__restrict__ rs,
                                                      const uint8_t *__restrict__ tile_body,
                                                      const int *__restrict__ body_tiles, int nb, DevState *ds,
                                                      unsigned int ncfl, DualPtrs dp) {
  __shared__ TileSmem sm;
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int b = (int)blockIdx.x;
  if (b < nb)
    stage_tile<STAGE, true, true>(k, c, nullptr, In, Out32, D, tag, sid, rs, tile_body, body_tiles, ds, false, ncfl,
                                  b, sm, dp);
  else
    stage_tile<STAGE, false, true>(k, c, nullptr, In, Out32, D, tag, sid, rs, tile_body, body_tiles, ds, false,
                                   ncfl, b - nb, sm, dp);
}

cudaError_t launch_dual_f32_one(const Consts &k, int stage, const float *In32, float *Out32, double *D,
                                const double *In64, double *Out64, const double *G, double *Q0,
                                const uint8_t *tag, const int *sid, const RStencil32 *rs, const uint8_t *tile_body,
                                const int *body_tiles, int body_cap, DevState *ds, bool pdl, cudaStream_t s) {
  const PertConsts c = pert_consts(k);
  const int nt = stage_tiles(k);
  const int nb = body_cap > 0 ? body_cap : 0;
  const unsigned int ncfl = (unsigned int)(nt + nb);
  DualPtrs dp;
  dp.In64 = In64;
  dp.Out64 = Out64;
  dp.G = G;
  dp.Q0 = Q0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned int)(nt + nb));
  cfg.blockDim = dim3(256);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
#define IBM_DUAL_ONE(S) \
  cudaLaunchKernelEx(&cfg, k_dual_f32_one<S>, k, c, In32, Out32, D, tag, sid, rs, tile_body, body_tiles, nb, ds, ncfl, dp)
  const cudaError_t e = stage == 1 ? IBM_DUAL_ONE(1) : stage == 2 ? IBM_DUAL_ONE(2) : IBM_DUAL_ONE(3);
#undef IBM_DUAL_ONE
  return e;
}

// Start of a physical step: one thread per FP64 word of the 4-plane state.
__global__ void __launch_bounds__(256) k_dual_levels(long long n, double idt, const double *__restrict__ A,
                                                     double *__restrict__ Wn, double *__restrict__ G,
                                                     const DevState *__restrict__ ds) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double wn = Wn[i], a = A[i];  // W^{n-1} and W^n of the new step
  G[i] = ds->steps > 0 ? (wn - 4.0 * a) * (0.5 * idt) : -a * idt;
  Wn[i] = a;
}

void launch_dual_levels(const Consts &k, const double *A, double *Wn, double *G, const DevState *ds, cudaStream_t s) {
  const long long n = 4 * k.plane;
  k_dual_levels<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, k.idt_phys, A, Wn, G, ds);
}

void launch_dual_f32(const Consts &k, int stage, const float *In32, float *Out32, double *D, const double *In64,
                     double *Out64, const double *G, double *Q0, const uint8_t *tag, const int *sid,
                     const RStencil32 *rs, const uint8_t *tile_body, const int *body_tiles, int body_cap,
                     DevState *ds, cudaStream_t s, cudaStream_t sb) {
  PertConsts c = pert_consts(k);
  const int nt = stage_tiles(k);
  const int nb = body_cap > 0 ? body_cap : 0;
  const unsigned int ncfl = (unsigned int)(nt + nb);
  DualPtrs dp;
  dp.In64 = In64;
  dp.Out64 = Out64;
  dp.G = G;
  dp.Q0 = Q0;
#define IBM_DUAL_PAIR(S)                                                                                          \
  do {                                                                                                            \
    if (nb)                                                                                                       \
      k_dual_f32<S, true><<<nb, 256, 0, sb>>>(k, c, In32, Out32, D, tag, sid, rs, tile_body, body_tiles, ds, ncfl, \
                                              dp);                                                                \
    k_dual_f32<S, false><<<nt, 256, 0, s>>>(k, c, In32, Out32, D, tag, sid, rs, tile_body, body_tiles, ds, ncfl,   \
                                            dp);                                                                  \
  } while (0)
  if (stage == 1) IBM_DUAL_PAIR(1);
  else if (stage == 2) IBM_DUAL_PAIR(2);
  else IBM_DUAL_PAIR(3);
#undef IBM_DUAL_PAIR
}

}  // namespace ibm
