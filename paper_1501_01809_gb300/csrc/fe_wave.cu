// Explicit linear wave steps with lumped mass (Sec. 6.3), fused around the pull action.
//
// State (phi, p) on the nodes of a P1 space, lumped mass m (the linear form v dx).  The paper's
// step is: phi -= dt/2 p; p += dt (K phi) / m, K phi the action of inner(grad v, grad phi) dx;
// p = sin(10 pi t) on Dirichlet nodes; phi -= dt/2 p.  p does not change between the second half
// step of one time step and the first half step of the next, so after one initial half step
// every time step is two launches:
//   1. the element kernel of the pull action (K_e phi_e per cell into staging; it reads phi);
//   2. one thread per node: y = sum of the node's staged contributions in incidence order,
//      p += dt y / m, the boundary value, then phi -= dt p (dt/2 in the last step).
// phi is only rewritten by launch 2, after every cell has read it.  Deterministic.
#include <cuda_runtime.h>

#include "fe_kernels.cuh"

namespace fe {
namespace {
using namespace kern;

__global__ void k_wave_half(int64_t n, double *__restrict__ phi, const double *__restrict__ p, double h) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    phi[i] -= h * p[i];
}

template <class Ops>
__global__ void k_wave_row(int64_t nrows, const int64_t *__restrict__ adjptr, const int32_t *__restrict__ adj,
                           const typename Ops::T *__restrict__ stage, const double *__restrict__ mass,
                           const uint8_t *__restrict__ is_bc, double pbc, double dt, double phi_dt,
                           double *__restrict__ p, double *__restrict__ phi) {
  using T = typename Ops::T;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nrows; r += (int64_t)gridDim.x * blockDim.x) {
    T s = Ops::zero();
    for (int64_t ai = adjptr[r]; ai < adjptr[r + 1]; ai++) s = Ops::add(s, stage[adj[ai]]);
    double pr = p[r] + dt * Ops::to_f64(s) / mass[r];
    if (is_bc && is_bc[r]) pr = pbc;
    p[r] = pr;
    phi[r] -= phi_dt * pr;
  }
}

template <int DIM, class Ops>
cudaError_t wave_run(const AsmArgs &a, void *stage_raw, const double *mass, const uint8_t *is_bc, double *p,
                     double t0, double dt, int nsteps, double (*bc_value)(double), cudaStream_t s) {
  using T = typename Ops::T;
  T *stage = static_cast<T *>(stage_raw);
  const unsigned gn = (unsigned)((a.nrows + 255) / 256 < 152 * 16 ? (a.nrows + 255) / 256 : 152 * 16);
  if (nsteps <= 0 || a.nrows == 0) return cudaSuccess;
  k_wave_half<<<gn, 256, 0, s>>>(a.nrows, a.y, p, 0.5 * dt);
  for (int k = 0; k < nsteps; k++) {
    if (a.ncell > 0)
      k_action_elem<DIM, 1, FE_FORM_LAPLACE, Ops><<<(unsigned)((a.ncell + kPushThreads - 1) / kPushThreads),
                                                   kPushThreads, 0, s>>>(a, stage);
    const double t = t0 + k * dt;
    k_wave_row<Ops><<<gn, 256, 0, s>>>(a.nrows, a.adjptr, a.adj, stage, mass, is_bc, bc_value(t), dt,
                                        k + 1 < nsteps ? dt : 0.5 * dt, p, a.y);
  }
  return cudaGetLastError();
}

}  // namespace

size_t wave_stage_bytes(int dim, int precision, int64_t ncell) {
  const size_t elem = precision == FE_PREC_F32X2 ? 2 * sizeof(float) : sizeof(double);
  return (size_t)ncell * (size_t)(dim + 1) * elem;
}

// a: the action's arguments with x = y = phi (the element kernel reads a.x, the row kernel writes
// a.y), adjacency of the (map, map) sparsity.  Returns cudaErrorInvalidValue for combinations
// that are not compiled (P1 Laplace, FP64 or double-float, triangles or tetrahedra).
cudaError_t launch_wave(const fe_form_desc &d, const AsmArgs &a, void *stage, const double *mass,
                        const uint8_t *is_bc, double *p, double t0, double dt, int nsteps,
                        double (*bc_value)(double), cudaStream_t s) {
  if (d.form != FE_FORM_LAPLACE || d.degree != 1) return cudaErrorInvalidValue;
  if (d.precision == FE_PREC_FP64) {
    if (d.dim == 2) return wave_run<2, OpsF64>(a, stage, mass, is_bc, p, t0, dt, nsteps, bc_value, s);
    if (d.dim == 3) return wave_run<3, OpsF64>(a, stage, mass, is_bc, p, t0, dt, nsteps, bc_value, s);
  } else if (d.precision == FE_PREC_F32X2) {
    if (d.dim == 2) return wave_run<2, OpsF32x2>(a, stage, mass, is_bc, p, t0, dt, nsteps, bc_value, s);
    if (d.dim == 3) return wave_run<3, OpsF32x2>(a, stage, mass, is_bc, p, t0, dt, nsteps, bc_value, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace fe
