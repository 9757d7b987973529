// Landmark-driven masses (Sec. IV-F): the RBF interpolant B of Eq. 17 and the
// smooth-particle masses S = N o B of Eq. 19.
//
// B(p) = sum_c lambda_c exp(-|p - p_c|^2 / sigma^2) over the m landmarks c,
// with the coefficients fixed by collocation at the landmarks (value 1 at
// every landmark: the strong weight the paper gives them), and clamped below
// at `floor` so that every mass stays positive. Without landmarks B = 1.
//   1. k_rbf_matrix: the m x m collocation matrix (FP64).
//   2. k_rbf_solve (one block): Cholesky factorisation in place, then the two
//      triangular solves for lambda (one warp); a matrix that is not positive
//      definite (repeated landmarks) sets a flag.
//   3. k_rbf_eval: B at every point (FP64, landmarks and lambda staged in
//      shared memory), times the NIV weight for S, rounded to FP32; the
//      result is then scaled to sum to `total`.
// m is at most FGA_MAX_LANDMARKS (the paper's landmark sets are small).
#include <cmath>
#include <cstring>
#include <vector>

#include "fga_internal.cuh"

namespace fga {
namespace {

constexpr int SOLVE_THREADS = 256;
constexpr unsigned FULL_MASK = 0xffffffffu;

__global__ void k_rbf_gather(const float* __restrict__ pts, const int64_t* __restrict__ idx, int m,
                             double* __restrict__ anchors) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < m)
    for (int k = 0; k < 3; ++k) anchors[3 * c + k] = (double)pts[3 * idx[c] + k];
}

__global__ void k_rbf_matrix(const double* __restrict__ anchors, int m, double inv_s2,
                             double* __restrict__ A) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)m * m) return;
  const int r = (int)(t / m), c = (int)(t % m);
  double d2 = 0;
  for (int k = 0; k < 3; ++k) {
    const double d = anchors[3 * r + k] - anchors[3 * c + k];
    d2 += d * d;
  }
  A[t] = exp(-d2 * inv_s2);
}

// Dot product of rows i and j of the lower triangle over columns [0, n),
// four independent partial sums (FP64 latency).
__device__ __forceinline__ double row_dot(const double* __restrict__ A, int m, int i, int j, int n) {
  double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  const double* a = A + (int64_t)i * m;
  const double* b = A + (int64_t)j * m;
  int k = 0;
  for (; k + 3 < n; k += 4) {
    s0 = fma(a[k], b[k], s0);
    s1 = fma(a[k + 1], b[k + 1], s1);
    s2 = fma(a[k + 2], b[k + 2], s2);
    s3 = fma(a[k + 3], b[k + 3], s3);
  }
  for (; k < n; ++k) s0 = fma(a[k], b[k], s0);
  return (s0 + s1) + (s2 + s3);
}

// One block: A = L L^T in place (lower triangle), then L z = 1 and
// L^T lambda = z. flag[0] = 1 if A is not positive definite.
__global__ void __launch_bounds__(SOLVE_THREADS) k_rbf_solve(double* __restrict__ A, int m,
                                                             double* __restrict__ lambda,
                                                             int* __restrict__ flag) {
  __shared__ double s_ljj;
  __shared__ int s_bad;
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  for (int j = 0; j < m; ++j) {
    if (threadIdx.x == 0) {
      const double s = A[(int64_t)j * m + j] - row_dot(A, m, j, j, j);
      if (!(s > 0)) s_bad = 1;
      s_ljj = s > 0 ? sqrt(s) : 1.0;
      A[(int64_t)j * m + j] = s_ljj;
    }
    __syncthreads();
    if (s_bad) break;
    const double ljj = s_ljj;
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x)
      A[(int64_t)i * m + j] = (A[(int64_t)i * m + j] - row_dot(A, m, i, j, j)) / ljj;
    __syncthreads();
  }
  if (s_bad) {
    if (threadIdx.x == 0) flag[0] = 1;
    return;
  }
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  // forward: z_i = (1 - sum_{k<i} L_ik z_k) / L_ii, z kept in lambda
  for (int i = 0; i < m; ++i) {
    double t = 0;
    for (int k = lane; k < i; k += 32) t = fma(A[(int64_t)i * m + k], lambda[k], t);
    for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(FULL_MASK, t, off);
    if (lane == 0) lambda[i] = (1.0 - t) / A[(int64_t)i * m + i];
    __syncwarp();
  }
  // backward: lambda_i = (z_i - sum_{k>i} L_ki lambda_k) / L_ii
  for (int i = m - 1; i >= 0; --i) {
    double t = 0;
    for (int k = i + 1 + lane; k < m; k += 32) t = fma(A[(int64_t)k * m + i], lambda[k], t);
    for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(FULL_MASK, t, off);
    if (lane == 0) lambda[i] = (lambda[i] - t) / A[(int64_t)i * m + i];
    __syncwarp();
  }
}

// out_i = max(B(p_i), floor) * (niv ? niv_i : 1), in FP32 before the final
// scaling. With m = 0, B = 1.
__global__ void k_rbf_eval(const float* __restrict__ pts, int64_t n, const double* __restrict__ anchors,
                           const double* __restrict__ lambda, int m, double inv_s2, double floor_v,
                           const float* __restrict__ niv, float* __restrict__ out) {
  extern __shared__ double s_an[];  // 4 per landmark: x, y, z, lambda
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    s_an[4 * c] = anchors[3 * c];
    s_an[4 * c + 1] = anchors[3 * c + 1];
    s_an[4 * c + 2] = anchors[3 * c + 2];
    s_an[4 * c + 3] = lambda[c];
  }
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double b = 1.0;
    if (m > 0) {
      const double x = pts[3 * i], y = pts[3 * i + 1], z = pts[3 * i + 2];
      b = 0;
      for (int c = 0; c < m; ++c) {
        const double dx = x - s_an[4 * c], dy = y - s_an[4 * c + 1], dz = z - s_an[4 * c + 2];
        b = fma(s_an[4 * c + 3], exp(-(dx * dx + dy * dy + dz * dz) * inv_s2), b);
      }
      b = b > floor_v ? b : floor_v;
    }
    out[i] = (float)(niv ? b * (double)niv[i] : b);
  }
}

}  // namespace
}  // namespace fga

using namespace fga;

extern "C" int fga_masses_landmarks(const float* pts, int64_t n, const int64_t* landmarks, int m,
                                    float sigma, float floor_v, int mode, int lattice, float a, float b,
                                    double total, float* masses_out, void* stream) {
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  if (n <= 0 || !pts || !masses_out || m < 0 || m > FGA_MAX_LANDMARKS || (m > 0 && !landmarks) ||
      !(sigma > 0.f) || !std::isfinite(sigma) || !(floor_v > 0.f) || !std::isfinite(floor_v) ||
      !(total > 0) || !std::isfinite(total) || (mode != FGA_MASS_RBF && mode != FGA_MASS_SPM) ||
      (mode == FGA_MASS_SPM && (lattice < 1 || lattice > 256 || !(b > a)))) {
    set_error("fga_masses_landmarks: bad arguments");
    return FGA_EINVAL;
  }
  for (int c = 0; c < m; ++c)
    if (landmarks[c] < 0 || landmarks[c] >= n) {
      set_error("fga_masses_landmarks: landmark " + std::to_string(c) + " is not a point index");
      return FGA_EINVAL;
    }
  Scratch sc(s);
  int64_t* d_idx = nullptr;
  double *anchors = nullptr, *A = nullptr, *lambda = nullptr;
  float *niv = nullptr, *tmp = nullptr;
  int* flag = nullptr;
  const int mm = m > 0 ? m : 1;
  if (sc.alloc(&d_idx, mm) || sc.alloc(&anchors, 3 * mm) || sc.alloc(&A, (size_t)mm * mm) ||
      sc.alloc(&lambda, mm) || sc.alloc(&flag, 1) || sc.alloc(&tmp, n))
    return FGA_ENOMEM;
  int rc = 0;
  if (mode == FGA_MASS_SPM) {
    if (sc.alloc(&niv, n)) return FGA_ENOMEM;
    if ((rc = masses_device(pts, n, FGA_MASS_NIV, lattice, a, b, 1.0, niv, s))) return rc;
  }
  const double inv_s2 = 1.0 / ((double)sigma * (double)sigma);
  FGA_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), s));
  if (m > 0) {
    FGA_CUDA_TRY(cudaMemcpyAsync(d_idx, landmarks, sizeof(int64_t) * m, cudaMemcpyHostToDevice, s));
    k_rbf_gather<<<(m + 127) / 128, 128, 0, s>>>(pts, d_idx, m, anchors);
    FGA_LAUNCH_CHECK("rbf_gather");
    const int64_t mm2 = (int64_t)m * m;
    k_rbf_matrix<<<(unsigned)((mm2 + 255) / 256), 256, 0, s>>>(anchors, m, inv_s2, A);
    FGA_LAUNCH_CHECK("rbf_matrix");
    k_rbf_solve<<<1, SOLVE_THREADS, 0, s>>>(A, m, lambda, flag);
    FGA_LAUNCH_CHECK("rbf_solve");
    int h = 0;
    if ((rc = read_flags(flag, 1, &h, s))) return rc;
    if (h) {
      set_error("fga_masses_landmarks: the collocation matrix is not positive definite "
                "(repeated or coincident landmarks)");
      return FGA_EINVAL;
    }
  }
  k_rbf_eval<<<grid_for(n), 256, (size_t)32 * mm, s>>>(pts, n, anchors, lambda, m, inv_s2, (double)floor_v,
                                                      niv, tmp);
  FGA_LAUNCH_CHECK("rbf_eval");
  return rescale_masses(tmp, n, total, masses_out, s);
}
