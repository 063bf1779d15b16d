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

// one launch of the pseudo stage of a case with the TVD-2 reconstruction and / or the quadratic IB / ghost
// reconstruction compiled in: body-tile slots [0, nb) first, then one block per tile (every launch form of such
// a case)
template <int STAGE, bool TVD, bool QUAD>
__global__ void __launch_bounds__(256) k_dual_f32_var(Consts k, PertConsts c, const float *__restrict__ In,
                                                      float *Out32, double *D, const uint8_t *__restrict__ tag,
                                                      const int *__restrict__ sid,
                                                      const RStencil32 *__restrict__ rs,
                                                      const uint8_t *__restrict__ tile_body,
                                                      const int *__restrict__ body_tiles, int nb, DevState *ds,
                                                      unsigned int ncfl, DualPtrs dp,
                                                      const RStencilQ *__restrict__ rsq) {
  __shared__ TileSmem sm;
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int b = (int)blockIdx.x;
  if (b < nb)
    stage_tile<STAGE, true, true, false, false, TVD, QUAD>(k, c, nullptr, In, Out32, D, tag, sid, rs, tile_body,
                                                           body_tiles, ds, false, ncfl, b, sm, dp, nullptr, rsq);
  else
    stage_tile<STAGE, false, true, false, false, TVD, QUAD>(k, c, nullptr, In, Out32, D, tag, sid, rs, tile_body,
                                                            body_tiles, ds, false, ncfl, b - nb, sm, dp, nullptr,
                                                            rsq);
}

cudaError_t launch_dual_f32_var(const Consts &k, int stage, const float *In32, float *Out32, double *D,
                                const double *In64, double *Out64, const double *G, double *Q0,
                                const uint8_t *tag, const int *sid, const RStencil32 *rs, const uint8_t *tile_body,
                                const int *body_tiles, int body_cap, DevState *ds, bool pdl, cudaStream_t s,
                                const RStencilQ *rsq) {
  if (k.quad && !rsq) return cudaErrorInvalidValue;  // the quadratic kernels read the second probes
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
#define IBM_DUAL_VAR(S, T, Q)                                                                                 \
  cudaLaunchKernelEx(&cfg, k_dual_f32_var<S, T, Q>, k, c, In32, Out32, D, tag, sid, rs, tile_body, body_tiles, nb, \
                     ds, ncfl, dp, rsq)
#define IBM_DUAL_VAR_S(S)                                                                                       \
  (k.tvd2 && k.quad ? IBM_DUAL_VAR(S, true, true)                                                              \
                    : k.tvd2 ? IBM_DUAL_VAR(S, true, false) : IBM_DUAL_VAR(S, false, true))
  const cudaError_t e = stage == 1 ? IBM_DUAL_VAR_S(1) : stage == 2 ? IBM_DUAL_VAR_S(2) : IBM_DUAL_VAR_S(3);
#undef IBM_DUAL_VAR_S
#undef IBM_DUAL_VAR
  return e;
}

// Dual-time pseudo stage over a block table: per entry the per-tile code --
// FP32 residual of the mirror, FP64 point-implicit update -- of the case the
// entry falls in, with its stage arrays and FP64 iterates rotated over the
// three pseudo stages (mirror -> F1 -> F2 -> mirror, D -> B -> C -> D).
// Body-tile entries of every case first.  A case alone runs it with a table
// of one entry (one block per tile), a group of dual-time cases with the
// group's table, so a case's results are the same bits alone and in a group.
// With programmatic dependent launch its blocks are resident while the
// previous pseudo stage's last blocks finish (they wait at the top for it to
// complete).
template <int STAGE>
__global__ void __launch_bounds__(256, 4) k_dual_f32_batch_one(const __grid_constant__ StageBatch b) {
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
    float *Out = STAGE == 1 ? sc.F1 : (STAGE == 2 ? sc.F2 : sc.M);
    DualPtrs dp;
    dp.In64 = STAGE == 1 ? sc.D : (STAGE == 2 ? sc.B : sc.C);
    dp.Out64 = STAGE == 1 ? sc.B : (STAGE == 2 ? sc.C : sc.D);
    dp.G = sc.G;
    dp.Q0 = sc.Q0;
    if (body)
      stage_tile<STAGE, true, true>(sc.k, sc.c, nullptr, In, Out, sc.D, sc.tag, sc.sid, sc.rs, sc.tile_body,
                                    sc.body_tiles, sc.ds, false, sc.ncfl, ee - start[q], sm, dp);
    else
      stage_tile<STAGE, false, true>(sc.k, sc.c, nullptr, In, Out, sc.D, sc.tag, sc.sid, sc.rs, sc.tile_body,
                                     sc.body_tiles, sc.ds, false, sc.ncfl, ee - start[q], sm, dp);
    __syncthreads();  // shared memory is reused by the next entry
  }
}

cudaError_t launch_dual_f32_batch_one(const StageBatch &b, int stage, int grid, bool pdl, cudaStream_t s) {
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
  if (stage == 1) return cudaLaunchKernelEx(&cfg, k_dual_f32_batch_one<1>, b);
  if (stage == 2) return cudaLaunchKernelEx(&cfg, k_dual_f32_batch_one<2>, b);
  return cudaLaunchKernelEx(&cfg, k_dual_f32_batch_one<3>, b);
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
                     DevState *ds, cudaStream_t s, cudaStream_t sb, const RStencilQ *rsq) {
  if (k.tvd2 || k.quad) {  // the variant kernel holds plain and body tiles: one launch on the case stream
    launch_dual_f32_var(k, stage, In32, Out32, D, In64, Out64, G, Q0, tag, sid, rs, tile_body, body_tiles, body_cap,
                        ds, false, s, rsq);
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
