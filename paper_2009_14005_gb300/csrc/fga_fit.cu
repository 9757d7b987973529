// fga_rigid_fit: one rigid fit of Algorithm 2 (Eqs. 14, 16) from given reduced
// sums, run by the same device code as every iteration of the registration
// loop (rigid_step_block: one matrix entry per lane, FP64). It lets the fit
// be checked on its own against an FP64 Kabsch step.
#include <cmath>

#include "fga_epi.cuh"

namespace fga {

// One block: the reductions into shared memory, then the fit on the state.
__global__ void __launch_bounds__(EPI_BS_MIN) k_rigid_fit(const double* __restrict__ red, int64_t M,
                                                          DevState* ds, EpiParams ep) {
  __shared__ double s_red[NRED];
  if (threadIdx.x < NRED) s_red[threadIdx.x] = red[threadIdx.x];
  __syncthreads();
  rigid_step_block(s_red, M, ds, ep, nullptr, 0ull);
}

}  // namespace fga

using namespace fga;

extern "C" int fga_rigid_fit(const double red[27], int64_t M, const double mu0[3], int dim, double R_out[9],
                             double t_out[3], void* stream) {
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  if (!red || !mu0 || !R_out || !t_out || M <= 0 || (dim != 2 && dim != 3)) {
    set_error("fga_rigid_fit: bad arguments");
    return FGA_EINVAL;
  }
  for (int k = 0; k < NRED; ++k)
    if (!std::isfinite(red[k])) {
      set_error("fga_rigid_fit: non-finite reduction");
      return FGA_EINVAL;
    }
  Scratch sc(s);
  DevState* ds = nullptr;
  double* d_buf = nullptr;  // the reductions (NRED) and mu0 (3)
  if (sc.alloc(&ds, 1) || sc.alloc(&d_buf, NRED + 3)) return FGA_ENOMEM;
  double h_buf[NRED + 3];
  for (int k = 0; k < NRED; ++k) h_buf[k] = red[k];
  for (int k = 0; k < 3; ++k) h_buf[NRED + k] = mu0[k];
  FGA_CUDA_TRY(cudaMemcpyAsync(d_buf, h_buf, sizeof(h_buf), cudaMemcpyHostToDevice, s));
  int rc = launch_state_init(ds, d_buf + NRED, s);
  if (rc) return rc;
  EpiParams ep{};
  ep.G = 0.f;
  ep.dt = 1.f;
  ep.eta = 0.f;
  ep.vmode = FGA_VEL_UNCONSTRAINED;
  ep.conv_tol = 0.0;
  ep.max_traj = 0;
  ep.inv_M = 1.0 / (double)M;
  ep.inv_dt = 1.0;
  ep.max_iter = 0;
  ep.dim = dim;
  k_rigid_fit<<<1, EPI_BS_MIN, 0, s>>>(d_buf, M, ds, ep);
  FGA_LAUNCH_CHECK("rigid_fit");
  DevState h;
  FGA_CUDA_TRY(cudaMemcpyAsync(&h, ds, sizeof(h), cudaMemcpyDeviceToHost, s));
  FGA_CUDA_TRY(cudaStreamSynchronize(s));
  for (int k = 0; k < 9; ++k) R_out[k] = h.R[k];
  for (int k = 0; k < 3; ++k) t_out[k] = h.t[k];
  return h.degenerate ? FGA_EDEGENERATE : FGA_OK;
}
