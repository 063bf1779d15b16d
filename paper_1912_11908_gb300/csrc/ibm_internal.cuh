// Internal declarations of the sm_103a immersed-boundary library (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ibm.h"

namespace ibm {

constexpr int NG = 3;  // halo / ghost layers for the five-point WENO stencil (Sec. 5)

enum : uint8_t { FLUID = 0, SOLID = 1, IB = 2, G1 = 3, G2 = 4, G3 = 5 };

// device-resident per-case scalars
struct DevState {
  double t;                      // time at the start of the current step
  double dt;                     // step size of the current step
  unsigned long long lmax_bits;  // max spectral radius (bits of a positive double)
  int count[4];                  // #IB, #G1, #G2, #G3
  int offset[5];                 // exclusive prefix of count; offset[4] = total
  int err;                       // bit 0: list capacity exceeded, bit 1: empty stencil
  int pad;
  double pos[2];                 // body displacement at the last classification
  double bbox[4];                // xmin, xmax, ymin, ymax of the current pose
  double force[4];               // Cd, Cl, Fx, Fy
  long long steps;
};

constexpr int ERR_CAPACITY = 1;
constexpr int ERR_STENCIL = 2;

// body motion (prescribed translation)
struct Motion {
  int kind;
  double amp[2], freq, vel[2];
};

// everything a kernel needs about the grid and the gas, passed by value
struct Consts {
  int nx, ny, pitch, rows;
  long long plane;  // pitch * rows
  double x0, y0, dx, dy, h, dmin;
  double gamma, R, cp, mu, kappa, pinf, prandtl, cfl, dt_fixed, ref_len;
  double uinf[2];
  double Uinf[4];   // free-stream conserved state
  double Hinf;      // free-stream total enthalpy
  int bc[4];
  Motion motion;
};

// geometry arrays (device)
struct Geom {
  int nv;
  const double *vref;   // 2*nv reference vertices
  double *vx, *vy;      // current pose
  const double *snx, *sny, *vnx, *vny;
};

__host__ __device__ inline long long cidx(const Consts &k, int i, int j) {
  return (long long)(j + NG) * k.pitch + (i + NG);
}

// motion state at time t
__device__ inline void motion_at(const Motion &m, double t, double X[2], double V[2], double A[2]) {
  X[0] = X[1] = V[0] = V[1] = A[0] = A[1] = 0.0;
  if (m.kind == IBM_MOTION_SIN) {
    const double w = 2.0 * 3.14159265358979323846 * m.freq;
    double s, c;
    sincos(w * t, &s, &c);
    for (int d = 0; d < 2; d++) {
      X[d] = m.amp[d] * s;
      V[d] = m.amp[d] * w * c;
      A[d] = -m.amp[d] * w * w * s;
    }
  } else if (m.kind == IBM_MOTION_CONST) {
    for (int d = 0; d < 2; d++) {
      X[d] = m.vel[d] * t;
      V[d] = m.vel[d];
    }
  }
}

// ---- launchers (geometry.cu) ----
void launch_normals(int nv, const double *v, double *snx, double *sny, double *vnx, double *vny, cudaStream_t s);
void launch_pose(const Consts &k, const Geom &g, DevState *ds, cudaStream_t s);
void launch_classify(const Consts &k, const Geom &g, uint8_t *solid, const DevState *ds, cudaStream_t s);
void launch_tags(const Consts &k, const uint8_t *solid, uint8_t *tag, int *blockcounts, DevState *ds, int cap,
                 ibm_stencil *st, cudaStream_t s, int *nlaunch);
void launch_stencils(const Consts &k, const Geom &g, const uint8_t *tag, ibm_stencil *st, int cap, DevState *ds,
                     cudaStream_t s);
void launch_forces_f64(const Consts &k, const Geom &g, const uint8_t *tag, const double *A, DevState *ds,
                       cudaStream_t s);

// ---- launchers (flow.cu) ----
void launch_dt(const Consts &k, const double *A, const uint8_t *tag, DevState *ds, cudaStream_t s, int *nlaunch);
void launch_recon_f64(const Consts &k, double *U, const ibm_stencil *st, int cap, const DevState *ds,
                      int stage, cudaStream_t s, int *nlaunch);
void launch_bc_f64(const Consts &k, double *U, cudaStream_t s);
void launch_stage_f64(const Consts &k, int stage, const double *Un, const double *In, double *Out,
                      const uint8_t *tag, const DevState *ds, cudaStream_t s);
void launch_step_end(const Consts &k, DevState *ds, cudaStream_t s);

// FP32-bulk path (flow32.cu)
void launch_to_pert(const Consts &k, const double *A, float *M, cudaStream_t s);
void launch_recon_f32(const Consts &k, float *U, double *A, const ibm_stencil *st, int cap, const DevState *ds,
                      int stage, cudaStream_t s, int *nlaunch);
void launch_bc_f32(const Consts &k, float *U, cudaStream_t s);
void launch_stage_f32(const Consts &k, int stage, const float *Mn, const float *In, float *Out, double *A,
                      const uint8_t *tag, const DevState *ds, cudaStream_t s);

}  // namespace ibm
