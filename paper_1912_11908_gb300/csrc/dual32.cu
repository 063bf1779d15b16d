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

// the same with the TVD-2 reconstruction compiled in (every launch form of a TVD-2 case)
template <int STAGE>
__global__ void __launch_bounds__(256) k_dual_f32_tvd(Consts k, PertConsts c, const float *__restrict__ In,
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
    stage_tile<STAGE, true, true, false, false, true>(k, c, nullptr, In, Out32, D, tag, sid, rs, tile_body,
                                                      body_tiles, ds, false, ncfl, b, sm, dp);
  else
    stage_tile<STAGE, false, true, false, false, true>(k, c, nullptr, In, Out32, D, tag, sid, rs, tile_body,
                                                       body_tiles, ds, false, ncfl, b - nb, sm, dp);
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
#define IBM_DUAL_ONE(K, S) \
  cudaLaunchKernelEx(&cfg, K<S>, k, c, In32, Out32, D, tag, sid, rs, tile_body, body_tiles, nb, ds, ncfl, dp)
  const cudaError_t e = k.tvd2 ? (stage == 1   ? IBM_DUAL_ONE(k_dual_f32_tvd, 1)
                                  : stage == 2 ? IBM_DUAL_ONE(k_dual_f32_tvd, 2)
                                               : IBM_DUAL_ONE(k_dual_f32_tvd, 3))
                               : (stage == 1   ? IBM_DUAL_ONE(k_dual_f32_one, 1)
                                  : stage == 2 ? IBM_DUAL_ONE(k_dual_f32_one, 2)
                                               : IBM_DUAL_ONE(k_dual_f32_one, 3));
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
  if (k.tvd2) {  // the TVD-2 kernel holds plain and body tiles: one launch on the case stream
    launch_dual_f32_one(k, stage, In32, Out32, D, In64, Out64, G, Q0, tag, sid, rs, tile_body, body_tiles, body_cap,
                        ds, false, s);
    return;
  }
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

// Self-check of f32_to_f64 / f64_to_f32 against the hardware conversions of
// this module: every FP32 bit pattern but the subnormals (which the FP32
// arithmetic flushes to zero), and 2^30 FP64 patterns from a counter-based
// generator (splitmix64) with exponents from below to above the FP32 range and
// one in four low words an exact rounding tie.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ bool same_double(double a, double b) {
  return (a != a && b != b) || __double_as_longlong(a) == __double_as_longlong(b);
}
__device__ __forceinline__ bool same_float(float a, float b) {
  return (a != a && b != b) || __float_as_uint(a) == __float_as_uint(b);
}

__global__ void __launch_bounds__(256) k_check_conversions(unsigned long long n64, unsigned long long *bad) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long nbad = 0;
  for (unsigned long long i = t; i < (1ull << 32); i += stride) {
    const unsigned int b = (unsigned int)i;
    if (((b >> 23) & 0xffu) == 0u && (b & 0x7fffffu) != 0u) continue;  // FP32 subnormal
    const float f = __uint_as_float(b);
    nbad += !same_double(f32_to_f64(f), (double)f);
  }
  for (unsigned long long i = t; i < n64; i += stride) {
    const unsigned long long r = mix64(i), q = mix64(i ^ 0x5851f42d4c957f2dull);
    const unsigned int e = 860u + (unsigned int)(r % 330u);  // binary64 exponent field 860 .. 1189
    const unsigned int hi = ((unsigned int)(r >> 32) & 0x80000000u) | (e << 20) | ((unsigned int)q & 0xfffffu);
    unsigned int lo = (unsigned int)(q >> 32);
    if ((r >> 20 & 3u) == 0u) lo = (lo & 0xe0000000u) | 0x10000000u;  // exact tie
    const double d = __hiloint2double((int)hi, (int)lo);
    nbad += !same_float(f64_to_f32(d), (float)d);
  }
  if (nbad) atomicAdd(bad, nbad);
}

cudaError_t check_float_conversions(unsigned long long *checked, unsigned long long *mismatched) {
  unsigned long long *bad = nullptr;
  cudaError_t e = cudaMalloc(&bad, sizeof *bad);
  if (e != cudaSuccess) return e;
  const unsigned long long n64 = 1ull << 30;
  e = cudaMemset(bad, 0, sizeof *bad);
  if (e == cudaSuccess) {
    k_check_conversions<<<152 * 8, 256>>>(n64, bad);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(mismatched, bad, sizeof *bad, cudaMemcpyDeviceToHost);
  cudaFree(bad);
  *checked = (1ull << 32) - 2ull * ((1ull << 23) - 1ull) + n64;
  return e;
}

}  // namespace ibm
