// Once-per-registration kernels: input checks, Appendix A normalisation,
// Sec. IV-F masses, bounding boxes, Morton keys, LSD radix sort and scans.
// All reductions use a fixed grid and a fixed combination order, so repeated
// runs on the same input give bit-identical results.
#include <algorithm>
#include <cfloat>

#include <math_constants.h>

#include "fga_internal.cuh"

namespace fga {

static constexpr int RB = 256;  // threads per reduction block
static constexpr unsigned FULL = 0xffffffffu;

static int red_grid(int64_t n) {
  int64_t g = (n + RB - 1) / RB;
  g = std::min<int64_t>(g, 2 * (int64_t)sm_count());
  return (int)std::max<int64_t>(g, 1);
}

// Sum of K doubles over the block; thread 0 gets the result in v.
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K]) {
  __shared__ double sh[RB / 32][K];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k)
    for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(FULL, v[k], off);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) sh[w][k] = v[k];
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      v[k] = lane < (RB / 32) ? sh[lane][k] : 0.0;
      for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(FULL, v[k], off);
    }
  }
  __syncthreads();
}

template <int K>
__device__ __forceinline__ void block_minmax(double (&mn)[K], double (&mx)[K]) {
  __shared__ double smn[RB / 32][K], smx[RB / 32][K];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k)
    for (int off = 16; off > 0; off >>= 1) {
      mn[k] = fmin(mn[k], __shfl_down_sync(FULL, mn[k], off));
      mx[k] = fmax(mx[k], __shfl_down_sync(FULL, mx[k], off));
    }
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) { smn[w][k] = mn[k]; smx[w][k] = mx[k]; }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      mn[k] = lane < (RB / 32) ? smn[lane][k] : DBL_MAX;
      mx[k] = lane < (RB / 32) ? smx[lane][k] : -DBL_MAX;
      for (int off = 16; off > 0; off >>= 1) {
        mn[k] = fmin(mn[k], __shfl_down_sync(FULL, mn[k], off));
        mx[k] = fmax(mx[k], __shfl_down_sync(FULL, mx[k], off));
      }
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------------ input checks

__global__ void k_check_finite(const float* __restrict__ p, int64_t n, int* flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(p[i])) atomicExch(flag, 1);
}

__global__ void k_check_masses(const float* __restrict__ m, int64_t n, int* flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(m[i]) || m[i] < 0.f) atomicExch(flag, 1);
}

int check_finite(const float* p, int64_t n, int* d_flag, cudaStream_t s) {
  k_check_finite<<<red_grid(n), RB, 0, s>>>(p, n, d_flag);
  FGA_LAUNCH_CHECK("check_finite");
  return FGA_OK;
}

int check_masses(const float* m, int64_t n, int* d_flag, cudaStream_t s) {
  k_check_masses<<<red_grid(n), RB, 0, s>>>(m, n, d_flag);
  FGA_LAUNCH_CHECK("check_masses");
  return FGA_OK;
}

// ------------------------------------------------------------------ Appendix A

// Per-block FP64 sums of x, y, z (A.1).
__global__ void k_sum3(const float* __restrict__ p, int64_t n, double* __restrict__ part) {
  double v[3] = {0, 0, 0};
  for (int64_t i = blockIdx.x * (int64_t)RB + threadIdx.x; i < n; i += (int64_t)gridDim.x * RB) {
    v[0] += p[3 * i];
    v[1] += p[3 * i + 1];
    v[2] += p[3 * i + 2];
  }
  block_sum<3>(v);
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; ++k) part[3 * blockIdx.x + k] = v[k];
}

// means: info[0..2] = X mean, info[3..5] = Y mean
__global__ void k_means(const double* __restrict__ px, int gx, int64_t N,
                        const double* __restrict__ py, int gy, int64_t M, double* info) {
  double v[6] = {0, 0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < gx; b += RB)
    for (int k = 0; k < 3; ++k) v[k] += px[3 * b + k];
  for (int b = threadIdx.x; b < gy; b += RB)
    for (int k = 0; k < 3; ++k) v[3 + k] += py[3 * b + k];
  block_sum<6>(v);
  if (threadIdx.x == 0) {
    for (int k = 0; k < 3; ++k) {
      info[k] = v[k] / (double)N;
      info[3 + k] = v[3 + k] / (double)M;
    }
  }
}

// Per-block min / max over all coordinates of a centred cloud (A.2).
__global__ void k_minmax_centred(const float* __restrict__ p, int64_t n,
                                 const double* __restrict__ mean, double* __restrict__ pmin,
                                 double* __restrict__ pmax) {
  double mn[1] = {DBL_MAX}, mx[1] = {-DBL_MAX};
  const double m0 = mean[0], m1 = mean[1], m2 = mean[2];
  for (int64_t i = blockIdx.x * (int64_t)RB + threadIdx.x; i < n; i += (int64_t)gridDim.x * RB) {
    double a = (double)p[3 * i] - m0, b = (double)p[3 * i + 1] - m1, c = (double)p[3 * i + 2] - m2;
    mn[0] = fmin(mn[0], fmin(a, fmin(b, c)));
    mx[0] = fmax(mx[0], fmax(a, fmax(b, c)));
  }
  block_minmax<1>(mn, mx);
  if (threadIdx.x == 0) {
    pmin[blockIdx.x] = mn[0];
    pmax[blockIdx.x] = mx[0];
  }
}

// info[6] = l, info[7] = s = (b - a)/(r - l); ok = r > l.
__global__ void k_range(const double* __restrict__ pmin, const double* __restrict__ pmax, int g,
                        float a, float b, double* info, int* ok) {
  double mn[1] = {DBL_MAX}, mx[1] = {-DBL_MAX};
  for (int i = threadIdx.x; i < g; i += RB) {
    mn[0] = fmin(mn[0], pmin[i]);
    mx[0] = fmax(mx[0], pmax[i]);
  }
  block_minmax<1>(mn, mx);
  if (threadIdx.x == 0) {
    double l = mn[0], r = mx[0];
    info[6] = l;
    info[7] = ((double)b - (double)a) / (r - l);
    *ok = (r > l) ? 1 : 0;
  }
}

// A.3: p^ = (p - mean - l) * s + a, FP64, rounded once to FP32.
__global__ void k_write_norm(const float* __restrict__ p, int64_t n, const double* __restrict__ info,
                             int which, float a, float* __restrict__ out) {
  const double* mean = info + 3 * which;
  const double l = info[6], sc = info[7], aa = (double)a;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 3 * n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int k = (int)(i % 3);
    out[i] = (float)(((double)p[i] - mean[k] - l) * sc + aa);
  }
}

int normalize_device(const float* X, int64_t N, const float* Y, int64_t M, float a, float b,
                     float* Xn, float* Yn, double* d_info, int* d_ok, cudaStream_t s) {
  const int gx = red_grid(N), gy = red_grid(M);
  double* part = nullptr;
  int rc = dev_alloc_n(&part, (size_t)3 * (gx + gy) + 2 * (gx + gy), s);
  if (rc) return rc;
  double* px = part;
  double* py = part + 3 * gx;
  double* pmin = part + 3 * (gx + gy);
  double* pmax = pmin + (gx + gy);
  k_sum3<<<gx, RB, 0, s>>>(X, N, px);
  FGA_LAUNCH_CHECK("sum3 X");
  k_sum3<<<gy, RB, 0, s>>>(Y, M, py);
  FGA_LAUNCH_CHECK("sum3 Y");
  k_means<<<1, RB, 0, s>>>(px, gx, N, py, gy, M, d_info);
  FGA_LAUNCH_CHECK("means");
  k_minmax_centred<<<gx, RB, 0, s>>>(X, N, d_info, pmin, pmax);
  FGA_LAUNCH_CHECK("minmax X");
  k_minmax_centred<<<gy, RB, 0, s>>>(Y, M, d_info + 3, pmin + gx, pmax + gx);
  FGA_LAUNCH_CHECK("minmax Y");
  k_range<<<1, RB, 0, s>>>(pmin, pmax, gx + gy, a, b, d_info, d_ok);
  FGA_LAUNCH_CHECK("range");
  k_write_norm<<<red_grid(3 * N), RB, 0, s>>>(X, N, d_info, 0, a, Xn);
  FGA_LAUNCH_CHECK("write_norm X");
  k_write_norm<<<red_grid(3 * M), RB, 0, s>>>(Y, M, d_info, 1, a, Yn);
  FGA_LAUNCH_CHECK("write_norm Y");
  dev_free(part, s);
  return FGA_OK;
}

// ------------------------------------------------------------------ Sec. IV-F masses

// Lattice cell of point i; with dim = 2 only x and y are binned (z cell 0).
__device__ __forceinline__ int niv_cell(const float* p, int64_t i, double a, double h, int L, int dim) {
  int c[3] = {0, 0, 0};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (k >= dim) break;
    double q = floor(((double)p[3 * i + k] - a) / h);
    q = q > (double)(L - 1) ? (double)(L - 1) : q;
    q = q < 0.0 ? 0.0 : q;
    c[k] = (int)q;
  }
  return (c[2] * L + c[1]) * L + c[0];
}

__global__ void k_niv_count(const float* __restrict__ p, int64_t n, double a, double h, int L, int dim,
                            unsigned* __restrict__ counts) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&counts[niv_cell(p, i, a, h, L, dim)], 1u);
}

// Eq. 18's covered fraction of a lattice cell, V(union of the balls of its
// points, inside the cell) / V(cell). The union is measured exactly along the
// cell's last axis (z in 3D, y in 2D) on NIV_COLS x NIV_COLS lines per 3D cell
// (NIV_STRIPS lines per 2D cell) placed at the midpoints of a regular grid
// across that axis: each ball that reaches a line cuts a chord, and the line
// contributes the length of the union of its chords inside the cell. The
// fraction is the mean covered length over the lines, divided by h. Ball
// centres are the points clamped to [a, b]; the radius is h / (2 D).
constexpr int NIV_COLS = 64, NIV_STRIPS = 1024, NIV_ZBITS = 10;

template <int DIM>
struct NivShape {
  static constexpr int Q = DIM == 3 ? NIV_COLS : NIV_STRIPS;
  static constexpr int LINES = DIM == 3 ? Q * Q : Q;
  static constexpr int TILES = LINES / 32;  // one warp task = 32 lines of one cell
};

// Sort key of point i: its cell above NIV_ZBITS bits of its position along
// the chord axis inside the cell, so that a cell's points are contiguous and
// ordered along the chords (the union below is exact in any order; this order
// lets one pass over the points follow a chain of overlapping chords).
__global__ void k_niv_key(const float* __restrict__ p, int64_t n, double a, double b, double h, int L,
                          int dim, unsigned* __restrict__ counts, unsigned long long* __restrict__ keys,
                          int* __restrict__ vals) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c = niv_cell(p, i, a, h, L, dim);
    atomicAdd(&counts[c], 1u);
    const int ca = dim == 3 ? c / (L * L) : (c / L) % L;  // cell index along the chord axis
    const double zc = fmin(fmax((double)p[3 * i + dim - 1], a), b);
    double q = floor((zc - __dadd_rn(a, __dmul_rn((double)ca, h))) / h * (double)(1 << NIV_ZBITS));
    q = fmin(fmax(q, 0.0), (double)((1 << NIV_ZBITS) - 1));
    keys[i] = ((unsigned long long)c << NIV_ZBITS) | (unsigned long long)q;
    vals[i] = (int)i;
  }
}

__global__ void k_niv_flag(const unsigned* __restrict__ counts, int64_t ncell, unsigned* __restrict__ flag) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell;
       c += (int64_t)gridDim.x * blockDim.x)
    flag[c] = counts[c] ? 1u : 0u;
}

// list[rank] = cell for every non-empty cell (rank = exclusive scan of the flags).
__global__ void k_niv_list(const unsigned* __restrict__ counts, const unsigned* __restrict__ rank,
                           int64_t ncell, unsigned* __restrict__ list) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell;
       c += (int64_t)gridDim.x * blockDim.x)
    if (counts[c]) list[rank[c]] = (unsigned)c;
}

// Clamped ball centres in sorted order: (x, y, z, 0).
__global__ void k_niv_gather(const float* __restrict__ p, const int* __restrict__ order, int64_t n,
                             float a, float b, float4* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = order[i];
    out[i] = make_float4(fminf(fmaxf(p[3 * j], a), b), fminf(fmaxf(p[3 * j + 1], a), b),
                         fminf(fmaxf(p[3 * j + 2], a), b), 0.f);
  }
}

// One warp per (non-empty cell, 32 lines) for the cells of ranks [r0, r1);
// each lane measures one line.
// Covered length of a line: starting from the cell's lower face s, repeated
// passes over the cell's points extend the reach e over every chord with
// lo <= e; a pass that extends nothing ends the component [s, e] and yields the
// lowest chord start above e, where the next component begins. Components are
// added in increasing order, as a sorted sweep would add them, and every
// endpoint is a chord end, so the length of the union does not depend on the
// order of the points. An FP32 distance test with a 1 % margin skips points
// that cannot reach the line; the chord itself is FP64 with explicitly
// rounded products (no contraction), the same arithmetic as a plain sweep.
// part[task] = sum over the warp's 32 lines, task = (rank - r0) * tiles + tile.
template <int DIM>
__global__ void __launch_bounds__(256) k_niv_cover(const float4* __restrict__ pts,
                                                   const unsigned* __restrict__ offs,
                                                   const unsigned* __restrict__ counts,
                                                   const unsigned* __restrict__ list,
                                                   const unsigned* __restrict__ nnz, int64_t r0,
                                                   int64_t r1, int L, double a, double h, double rr,
                                                   double* __restrict__ part) {
  using S = NivShape<DIM>;
  const int lane = threadIdx.x & 31;
  const int64_t rend = r1 < (int64_t)(*nnz) ? r1 : (int64_t)(*nnz);
  const int64_t ntask = rend > r0 ? (rend - r0) * S::TILES : 0;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const double dlt = h / (double)S::Q;
  const float rrf = (float)(rr * 1.01);
  for (int64_t task = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; task < ntask;
       task += nwarp) {
    const unsigned c = list[r0 + task / S::TILES];
    const int ln = (int)(task % S::TILES) * 32 + lane;
    const unsigned first = offs[c], nc = counts[c];
    const int cx = (int)(c % (unsigned)L), cy = (int)((c / (unsigned)L) % (unsigned)L);
    const int cz = DIM == 3 ? (int)(c / ((unsigned)L * (unsigned)L)) : 0;
    const double lox = __dadd_rn(a, __dmul_rn((double)cx, h));
    const double loy = __dadd_rn(a, __dmul_rn((double)cy, h));
    const double u = __dadd_rn(lox, __dmul_rn((double)(ln % S::Q) + 0.5, dlt));
    const double v = DIM == 3 ? __dadd_rn(loy, __dmul_rn((double)(ln / S::Q) + 0.5, dlt)) : 0.0;
    const double clo = DIM == 3 ? __dadd_rn(a, __dmul_rn((double)cz, h)) : loy;
    const double chi = clo + h;
    const float uf = (float)u, vf = (float)v;
    double s = clo, total = 0.0;
    for (;;) {
      double e = s, nxt;
      bool grew;
      do {
        grew = false;
        nxt = CUDART_INF;
        for (unsigned t = 0; t < nc; ++t) {
          const float4 q = pts[first + t];
          const float dxf = uf - q.x;
          float d2f = dxf * dxf;
          if (DIM == 3) {
            const float dyf = vf - q.y;
            d2f = __fadd_rn(d2f, __fmul_rn(dyf, dyf));
          }
          if (d2f >= rrf) continue;
          const double dx = u - (double)q.x;
          double d2 = __dmul_rn(dx, dx);
          if (DIM == 3) {
            const double dy = v - (double)q.y;
            d2 = __dadd_rn(d2, __dmul_rn(dy, dy));
          }
          if (d2 >= rr) continue;
          const double w = sqrt(rr - d2);
          const double zc = DIM == 3 ? (double)q.z : (double)q.y;
          const double lo = fmax(zc - w, clo), hi = fmin(zc + w, chi);
          if (!(hi > lo)) continue;
          if (lo <= e) {
            if (hi > e) {
              e = hi;
              grew = true;
            }
          } else {
            nxt = fmin(nxt, lo);
          }
        }
      } while (grew);
      total += e - s;
      if (nxt == CUDART_INF) break;
      s = nxt;
    }
    for (int off = 16; off > 0; off >>= 1) total += __shfl_down_sync(FULL, total, off);
    if (lane == 0) part[task] = total;
  }
}

// Non-empty cells of ranks [r0, r1): fraction = (sum of the cell's tiles, in
// tile order) / (lines * h), weight w = 1 / fraction.
__global__ void k_niv_cellw(const unsigned* __restrict__ list, const unsigned* __restrict__ nnz,
                            int64_t r0, int64_t r1, const double* __restrict__ cover, int tiles,
                            int lines, double h, double* __restrict__ w) {
  const int64_t rend = r1 < (int64_t)(*nnz) ? r1 : (int64_t)(*nnz);
  for (int64_t r = r0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rend;
       r += (int64_t)gridDim.x * blockDim.x) {
    double sum = 0.0;
    for (int t = 0; t < tiles; ++t) sum += cover[(r - r0) * tiles + t];
    const double frac = sum / ((double)lines * h);
    w[list[r]] = frac > 0.0 ? 1.0 / frac : 0.0;
  }
}

// Per-block sums of count * w over the non-empty cells.
__global__ void k_niv_wsum(const unsigned* __restrict__ counts, int64_t ncell,
                           const double* __restrict__ w, double* __restrict__ part) {
  double v[1] = {0};
  for (int64_t c = blockIdx.x * (int64_t)RB + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * RB)
    if (counts[c]) v[0] += (double)counts[c] * w[c];
  block_sum<1>(v);
  if (threadIdx.x == 0) part[blockIdx.x] = v[0];
}

__global__ void k_sum_parts(const double* __restrict__ part, int g, double* out) {
  double v[1] = {0};
  for (int i = threadIdx.x; i < g; i += RB) v[0] += part[i];
  block_sum<1>(v);
  if (threadIdx.x == 0) *out = v[0];
}

__global__ void k_niv_assign(const float* __restrict__ p, int64_t n, double a, double h, int L, int dim,
                             const double* __restrict__ w, const double* __restrict__ wsum,
                             double total, float* __restrict__ out) {
  const double inv = total / *wsum;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)(w[niv_cell(p, i, a, h, L, dim)] * inv);
}

// Inverse-density weight of every point from its k-th nearest other point:
// w_i = max(r_k(i), r_min)^dim (brute force over tiles of all points in shared
// memory; the k smallest squared distances of a point are kept sorted in
// registers by an unrolled insertion).
template <int K>
__global__ void __launch_bounds__(256) k_knn_weight(const float* __restrict__ p, int64_t n, int dim,
                                                    float rmin, float* __restrict__ w) {
  __shared__ float4 tile[256];
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool valid = i < n;
  const float x = valid ? p[3 * i] : 0.f, y = valid ? p[3 * i + 1] : 0.f;
  const float z = (valid && dim == 3) ? p[3 * i + 2] : 0.f;
  float best[K];
#pragma unroll
  for (int q = 0; q < K; ++q) best[q] = FLT_MAX;
  for (int64_t base = 0; base < n; base += 256) {
    const int64_t j = base + threadIdx.x;
    tile[threadIdx.x] = j < n ? make_float4(p[3 * j], p[3 * j + 1], dim == 3 ? p[3 * j + 2] : 0.f, 0.f)
                              : make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    const int cnt = n - base < 256 ? (int)(n - base) : 256;
    for (int c = 0; c < cnt; ++c) {
      const float4 q4 = tile[c];
      const float dx = q4.x - x, dy = q4.y - y, dz = q4.z - z;
      const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      if (d2 < best[K - 1] && base + c != i) {
        // new[q] = max(old[q-1], min(old[q], d2)), from the top down
#pragma unroll
        for (int q = K - 1; q > 0; --q) best[q] = fmaxf(best[q - 1], fminf(best[q], d2));
        best[0] = fminf(best[0], d2);
      }
    }
    __syncthreads();
  }
  if (valid) {
    const float r = fmaxf(sqrtf(best[K - 1]), rmin);
    w[i] = dim == 3 ? r * r * r : r * r;
  }
}

// (x, y) pairs -> (x, y, 0): a planar cloud in the plane z = 0.
__global__ void k_embed2(const float* __restrict__ in, int64_t n, float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    out[3 * i] = in[2 * i];
    out[3 * i + 1] = in[2 * i + 1];
    out[3 * i + 2] = 0.f;
  }
}

__global__ void k_fill(float* __restrict__ out, int64_t n, float v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = v;
}

int embed_planar(const float* in2, int64_t n, float* out3, cudaStream_t s) {
  k_embed2<<<red_grid(n), RB, 0, s>>>(in2, n, out3);
  FGA_LAUNCH_CHECK("embed2");
  return FGA_OK;
}

int masses_device(const float* pts, int64_t n, int mode, int lattice, float a, float b,
                  double total, float* out, cudaStream_t s, int dim) {
  if (mode == FGA_MASS_KNN) {
    float* w = nullptr;
    int rc = dev_alloc_n(&w, (size_t)n, s);
    if (rc) return rc;
    const float rmin = 1e-6f * (b - a);
    const unsigned g = (unsigned)((n + 255) / 256);
    if (lattice == 8)
      k_knn_weight<8><<<g, 256, 0, s>>>(pts, n, dim, rmin, w);
    else if (lattice == 32)
      k_knn_weight<32><<<g, 256, 0, s>>>(pts, n, dim, rmin, w);
    else
      k_knn_weight<16><<<g, 256, 0, s>>>(pts, n, dim, rmin, w);
    FGA_LAUNCH_CHECK("knn_weight");
    rc = rescale_masses(w, n, total, out, s);
    dev_free(w, s);
    return rc;
  }
  if (mode == FGA_MASS_UNIFORM) {
    k_fill<<<red_grid(n), RB, 0, s>>>(out, n, (float)(total / (double)n));
    FGA_LAUNCH_CHECK("fill");
    return FGA_OK;
  }
  const int L = lattice;
  const int64_t ncell = dim == 2 ? (int64_t)L * L : (int64_t)L * L * L;
  const double h = ((double)b - (double)a) / (double)L;
  // Eq. 18 with d = D: balls of radius (b-a)/(2 D rho); discs for D = 2
  const double rad = ((double)b - (double)a) / (2.0 * (double)dim * (double)L);
  const double rr = rad * rad;
  const int tiles = dim == 2 ? NivShape<2>::TILES : NivShape<3>::TILES;
  const int lines = dim == 2 ? NivShape<2>::LINES : NivShape<3>::LINES;
  int cell_bits = 1;
  while (cell_bits < 40 && ((int64_t)1 << cell_bits) < ncell) ++cell_bits;
  const int gc = red_grid(ncell);
  // non-empty cells are measured in chunks of at most NIV_CHUNK cells, so the
  // per-task sums stay small whatever the lattice
  constexpr int64_t NIV_CHUNK = 32768;
  const int64_t cells_max = std::min<int64_t>(n, ncell);
  const int64_t chunk = std::min<int64_t>(cells_max, NIV_CHUNK);
  unsigned* u32 = nullptr;        // counts, offs, flags, ranks, list, nnz
  unsigned long long* keys = nullptr;
  int* vals = nullptr;
  float4* centres = nullptr;
  double* dbl = nullptr;          // w (ncell), cover (chunk * tiles), part (gc), wsum
  int rc = dev_alloc_n(&u32, (size_t)5 * ncell + 1, s);
  if (!rc) rc = dev_alloc_n(&keys, (size_t)2 * n, s);
  if (!rc) rc = dev_alloc_n(&vals, (size_t)2 * n, s);
  if (!rc) rc = dev_alloc_n(&centres, (size_t)n, s);
  if (!rc) rc = dev_alloc_n(&dbl, (size_t)ncell + chunk * tiles + gc + 1, s);
  if (rc) {
    dev_free(u32, s);
    dev_free(keys, s);
    dev_free(vals, s);
    dev_free(centres, s);
    dev_free(dbl, s);
    return rc;
  }
  unsigned *counts = u32, *offs = u32 + ncell, *flag = u32 + 2 * ncell, *rank = u32 + 3 * ncell;
  unsigned *list = u32 + 4 * ncell, *nnz = u32 + 5 * ncell;
  double *w = dbl, *cover = dbl + ncell, *part = cover + chunk * tiles, *wsum = part + gc;
  FGA_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(unsigned) * ncell, s));
  k_niv_key<<<red_grid(n), RB, 0, s>>>(pts, n, (double)a, (double)b, h, L, dim, counts, keys, vals);
  FGA_LAUNCH_CHECK("niv_key");
  rc = radix_sort_pairs(keys, vals, keys + n, vals + n, n, cell_bits + NIV_ZBITS, s);
  if (!rc) rc = scan_exclusive(counts, offs, ncell, nullptr, s);
  if (!rc) {
    k_niv_flag<<<gc, RB, 0, s>>>(counts, ncell, flag);
    FGA_LAUNCH_CHECK("niv_flag");
    rc = scan_exclusive(flag, rank, ncell, nnz, s);
  }
  if (!rc) {
    k_niv_list<<<gc, RB, 0, s>>>(counts, rank, ncell, list);
    FGA_LAUNCH_CHECK("niv_list");
    k_niv_gather<<<red_grid(n), RB, 0, s>>>(pts, vals, n, a, b, centres);
    FGA_LAUNCH_CHECK("niv_gather");
    const unsigned gcov = (unsigned)(8 * sm_count());
    for (int64_t r0 = 0; r0 < cells_max; r0 += chunk) {
      const int64_t r1 = std::min<int64_t>(r0 + chunk, cells_max);
      if (dim == 2)
        k_niv_cover<2><<<gcov, 256, 0, s>>>(centres, offs, counts, list, nnz, r0, r1, L, (double)a, h,
                                            rr, cover);
      else
        k_niv_cover<3><<<gcov, 256, 0, s>>>(centres, offs, counts, list, nnz, r0, r1, L, (double)a, h,
                                            rr, cover);
      FGA_LAUNCH_CHECK("niv_cover");
      k_niv_cellw<<<red_grid(r1 - r0), RB, 0, s>>>(list, nnz, r0, r1, cover, tiles, lines, h, w);
      FGA_LAUNCH_CHECK("niv_cellw");
    }
    k_niv_wsum<<<gc, RB, 0, s>>>(counts, ncell, w, part);
    FGA_LAUNCH_CHECK("niv_wsum_blocks");
    k_sum_parts<<<1, RB, 0, s>>>(part, gc, wsum);
    FGA_LAUNCH_CHECK("niv_wsum");
    k_niv_assign<<<red_grid(n), RB, 0, s>>>(pts, n, (double)a, h, L, dim, w, wsum, total, out);
    FGA_LAUNCH_CHECK("niv_assign");
  }
  dev_free(u32, s);
  dev_free(keys, s);
  dev_free(vals, s);
  dev_free(centres, s);
  dev_free(dbl, s);
  return rc;
}

__global__ void k_sum1(const float* __restrict__ m, int64_t n, double* __restrict__ part) {
  double v[1] = {0};
  for (int64_t i = blockIdx.x * (int64_t)RB + threadIdx.x; i < n; i += (int64_t)gridDim.x * RB)
    v[0] += m[i];
  block_sum<1>(v);
  if (threadIdx.x == 0) part[blockIdx.x] = v[0];
}

__global__ void k_scale(const float* __restrict__ in, int64_t n, const double* __restrict__ sum,
                        double total, float* __restrict__ out) {
  const double f = total / *sum;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)((double)in[i] * f);
}

int rescale_masses(const float* in, int64_t n, double total, float* out, cudaStream_t s) {
  const int g = red_grid(n);
  double* part = nullptr;
  int rc = dev_alloc_n(&part, (size_t)g + 1, s);
  if (rc) return rc;
  k_sum1<<<g, RB, 0, s>>>(in, n, part);
  FGA_LAUNCH_CHECK("mass_sum");
  k_sum_parts<<<1, RB, 0, s>>>(part, g, part + g);
  FGA_LAUNCH_CHECK("mass_total");
  k_scale<<<red_grid(n), RB, 0, s>>>(in, n, part + g, total, out);
  FGA_LAUNCH_CHECK("mass_scale");
  dev_free(part, s);
  return FGA_OK;
}

// ------------------------------------------------------------------ bounding box

__global__ void k_bbox_part(const float* __restrict__ p, int64_t n, double* __restrict__ pmin,
                            double* __restrict__ pmax) {
  double mn[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, mx[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
  for (int64_t i = blockIdx.x * (int64_t)RB + threadIdx.x; i < n; i += (int64_t)gridDim.x * RB)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double v = p[3 * i + k];
      mn[k] = fmin(mn[k], v);
      mx[k] = fmax(mx[k], v);
    }
  block_minmax<3>(mn, mx);
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; ++k) {
      pmin[3 * blockIdx.x + k] = mn[k];
      pmax[3 * blockIdx.x + k] = mx[k];
    }
}

__global__ void k_bbox_final(const double* __restrict__ pmin, const double* __restrict__ pmax,
                             int g, float* lo, float* hi) {
  double mn[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, mx[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
  for (int b = threadIdx.x; b < g; b += RB)
    for (int k = 0; k < 3; ++k) {
      mn[k] = fmin(mn[k], pmin[3 * b + k]);
      mx[k] = fmax(mx[k], pmax[3 * b + k]);
    }
  block_minmax<3>(mn, mx);
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; ++k) {
      lo[k] = (float)mn[k];  // exact: the extremes are input floats
      hi[k] = (float)mx[k];
    }
}

int bbox_xyz(const float* p, int64_t n, float* d_lo, float* d_hi, cudaStream_t s) {
  const int g = red_grid(n);
  double* part = nullptr;
  int rc = dev_alloc_n(&part, (size_t)6 * g, s);
  if (rc) return rc;
  k_bbox_part<<<g, RB, 0, s>>>(p, n, part, part + 3 * g);
  FGA_LAUNCH_CHECK("bbox_part");
  k_bbox_final<<<1, RB, 0, s>>>(part, part + 3 * g, g, d_lo, d_hi);
  FGA_LAUNCH_CHECK("bbox_final");
  dev_free(part, s);
  return FGA_OK;
}

// ------------------------------------------------------------------ Morton keys

// Integer cell of x along one axis at `bits` levels: floor((x - lo)/(hi - lo) 2^bits),
// clamped; an axis of zero extent maps to 0. Computed in FP64: x - lo is exact for
// float inputs, and the division is correctly rounded.
__device__ __forceinline__ unsigned axis_cell(float x, float lo, float hi, int bits) {
  const double ext = (double)hi - (double)lo;
  if (!(ext > 0.0)) return 0u;
  const double q = floor(((double)x - (double)lo) / ext * (double)(1u << bits));
  const double top = (double)((1u << bits) - 1u);
  return (unsigned)(q < 0.0 ? 0.0 : (q > top ? top : q));
}

// Bit i of each axis cell goes to key bit 3i (x), 3i+1 (y), 3i+2 (z), so the
// three key bits 3(bits-L) .. 3(bits-L)+2 are the octant at level L.
__global__ void k_morton(const float* __restrict__ p, int64_t n, const float* __restrict__ lo,
                         const float* __restrict__ hi, int bits,
                         unsigned long long* __restrict__ keys, int* __restrict__ idx) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    unsigned q[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) q[k] = axis_cell(p[3 * i + k], lo[k], hi[k], bits);
    unsigned long long key = 0;
    for (int bit = 0; bit < bits; ++bit)
#pragma unroll
      for (int k = 0; k < 3; ++k)
        key |= (unsigned long long)((q[k] >> bit) & 1u) << (3 * bit + k);
    keys[i] = key;
    idx[i] = (int)i;
  }
}

int morton_keys(const float* xyz, int64_t n, const float* d_lo, const float* d_hi, int bits,
                unsigned long long* keys, int* idx, cudaStream_t s) {
  k_morton<<<red_grid(n), RB, 0, s>>>(xyz, n, d_lo, d_hi, bits, keys, idx);
  FGA_LAUNCH_CHECK("morton");
  return FGA_OK;
}

// ------------------------------------------------------------------ scan

static constexpr int SCAN_BS = 256, SCAN_IPT = 4, SCAN_TILE = SCAN_BS * SCAN_IPT;

// Exclusive scan of one tile in place in registers; returns the tile total.
__device__ __forceinline__ unsigned tile_scan(unsigned (&v)[SCAN_IPT]) {
  __shared__ unsigned wsum[SCAN_BS / 32];
  __shared__ unsigned total;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned local = 0;
#pragma unroll
  for (int k = 0; k < SCAN_IPT; ++k) {
    unsigned x = v[k];
    v[k] = local;
    local += x;
  }
  unsigned inc = local;
  for (int off = 1; off < 32; off <<= 1) {
    unsigned y = __shfl_up_sync(FULL, inc, off);
    if (lane >= off) inc += y;
  }
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  if (w == 0) {
    unsigned x = lane < SCAN_BS / 32 ? wsum[lane] : 0u;
    unsigned ix = x;
    for (int off = 1; off < 32; off <<= 1) {
      unsigned y = __shfl_up_sync(FULL, ix, off);
      if (lane >= off) ix += y;
    }
    if (lane < SCAN_BS / 32) wsum[lane] = ix - x;
    if (lane == SCAN_BS / 32 - 1) total = ix;
  }
  __syncthreads();
  const unsigned base = wsum[w] + inc - local;
#pragma unroll
  for (int k = 0; k < SCAN_IPT; ++k) v[k] += base;
  unsigned t = total;
  __syncthreads();
  return t;
}

__global__ void k_scan_tiles(const unsigned* __restrict__ in, unsigned* __restrict__ out, int64_t n,
                             unsigned* __restrict__ bsum) {
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_IPT;
  unsigned v[SCAN_IPT];
#pragma unroll
  for (int k = 0; k < SCAN_IPT; ++k) v[k] = base + k < n ? in[base + k] : 0u;
  unsigned t = tile_scan(v);
#pragma unroll
  for (int k = 0; k < SCAN_IPT; ++k)
    if (base + k < n) out[base + k] = v[k];
  if (threadIdx.x == 0) bsum[blockIdx.x] = t;
}

// Single block: exclusive scan of the tile totals (any count), grand total.
__global__ void k_scan_bsums(unsigned* __restrict__ bsum, int64_t nb, unsigned* __restrict__ total) {
  unsigned carry = 0;
  for (int64_t t0 = 0; t0 < nb; t0 += SCAN_TILE) {
    const int64_t base = t0 + (int64_t)threadIdx.x * SCAN_IPT;
    unsigned v[SCAN_IPT];
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k) v[k] = base + k < nb ? bsum[base + k] : 0u;
    unsigned t = tile_scan(v);
#pragma unroll
    for (int k = 0; k < SCAN_IPT; ++k)
      if (base + k < nb) bsum[base + k] = v[k] + carry;
    carry += t;
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void k_scan_add(unsigned* __restrict__ out, int64_t n, const unsigned* __restrict__ bsum) {
  const unsigned add = bsum[blockIdx.x];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  for (int k = threadIdx.x; k < SCAN_TILE; k += SCAN_BS)
    if (base + k < n) out[base + k] += add;
}

int scan_exclusive(const unsigned* in, unsigned* out, int64_t n, unsigned* d_total, cudaStream_t s) {
  const int64_t nb = std::max<int64_t>((n + SCAN_TILE - 1) / SCAN_TILE, 1);
  unsigned* bsum = nullptr;
  int rc = dev_alloc_n(&bsum, (size_t)nb, s);
  if (rc) return rc;
  k_scan_tiles<<<(unsigned)nb, SCAN_BS, 0, s>>>(in, out, n, bsum);
  FGA_LAUNCH_CHECK("scan_tiles");
  k_scan_bsums<<<1, SCAN_BS, 0, s>>>(bsum, nb, d_total);
  FGA_LAUNCH_CHECK("scan_bsums");
  k_scan_add<<<(unsigned)nb, SCAN_BS, 0, s>>>(out, n, bsum);
  FGA_LAUNCH_CHECK("scan_add");
  dev_free(bsum, s);
  return FGA_OK;
}

// ------------------------------------------------------------------ radix sort

static constexpr int RS_BS = 256, RS_IPT = 8, RS_TILE = RS_BS * RS_IPT, RS_WARPS = RS_BS / 32;

__global__ void k_rs_hist(const unsigned long long* __restrict__ keys, int64_t n, int shift,
                          unsigned* __restrict__ hist, int64_t ntiles) {
  __shared__ unsigned h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll
  for (int it = 0; it < RS_IPT; ++it) {
    const int64_t i = base + (int64_t)it * RS_BS + threadIdx.x;
    if (i < n) atomicAdd(&h[(unsigned)(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: within a tile, keys keep their index order (rounds in order,
// warps in order, lanes ranked by __match_any_sync); tiles are ordered by the
// digit-major / tile-minor scan of the histograms.
__global__ void k_rs_scatter(const unsigned long long* __restrict__ kin, const int* __restrict__ vin,
                             unsigned long long* __restrict__ kout, int* __restrict__ vout,
                             int64_t n, int shift, const unsigned* __restrict__ offs, int64_t ntiles) {
  __shared__ unsigned run[256];
  __shared__ unsigned wcnt[RS_WARPS][256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  run[threadIdx.x] = offs[(int64_t)threadIdx.x * ntiles + blockIdx.x];
  const int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int it = 0; it < RS_IPT; ++it) {
    const int64_t i = base + (int64_t)it * RS_BS + threadIdx.x;
    const bool valid = i < n;
    unsigned long long key = valid ? kin[i] : 0ull;
    const unsigned digit = valid ? ((unsigned)(key >> shift) & 255u) : 256u;
#pragma unroll
    for (int ww = 0; ww < RS_WARPS; ++ww) wcnt[ww][threadIdx.x] = 0u;
    __syncthreads();
    const unsigned peers = __match_any_sync(FULL, digit);
    const unsigned rank = __popc(peers & lt_mask);
    const int leader = __ffs(peers) - 1;
    if (valid && lane == leader) wcnt[w][digit] = __popc(peers);
    __syncthreads();
    unsigned acc = 0;
#pragma unroll
    for (int ww = 0; ww < RS_WARPS; ++ww) {
      unsigned c = wcnt[ww][threadIdx.x];
      wcnt[ww][threadIdx.x] = acc;
      acc += c;
    }
    __syncthreads();
    if (valid) {
      const unsigned pos = run[digit] + wcnt[w][digit] + rank;
      kout[pos] = key;
      vout[pos] = vin[i];
    }
    __syncthreads();
    run[threadIdx.x] += acc;
    __syncthreads();
  }
}

int radix_sort_pairs(unsigned long long* keys, int* vals, unsigned long long* keys_tmp,
                     int* vals_tmp, int64_t n, int bits, cudaStream_t s) {
  if (n <= 1) return FGA_OK;
  const int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
  unsigned* hist = nullptr;
  int rc = dev_alloc_n(&hist, (size_t)2 * 256 * ntiles, s);
  if (rc) return rc;
  unsigned* offs = hist + 256 * ntiles;
  unsigned long long *ka = keys, *kb = keys_tmp;
  int *va = vals, *vb = vals_tmp;
  int passes = 0;
  for (int shift = 0; shift < bits; shift += 8) {
    k_rs_hist<<<(unsigned)ntiles, RS_BS, 0, s>>>(ka, n, shift, hist, ntiles);
    FGA_LAUNCH_CHECK("rs_hist");
    rc = scan_exclusive(hist, offs, 256 * ntiles, nullptr, s);
    if (rc) return rc;
    k_rs_scatter<<<(unsigned)ntiles, RS_BS, 0, s>>>(ka, va, kb, vb, n, shift, offs, ntiles);
    FGA_LAUNCH_CHECK("rs_scatter");
    std::swap(ka, kb);
    std::swap(va, vb);
    ++passes;
  }
  if (passes & 1) {
    FGA_CUDA_TRY(cudaMemcpyAsync(keys, ka, sizeof(unsigned long long) * n, cudaMemcpyDeviceToDevice, s));
    FGA_CUDA_TRY(cudaMemcpyAsync(vals, va, sizeof(int) * n, cudaMemcpyDeviceToDevice, s));
  }
  dev_free(hist, s);
  return FGA_OK;
}

// ------------------------------------------------------------------ centroid

__global__ void k_sum4(const float4* __restrict__ p, int64_t n, double* __restrict__ part) {
  double v[3] = {0, 0, 0};
  for (int64_t i = blockIdx.x * (int64_t)RB + threadIdx.x; i < n; i += (int64_t)gridDim.x * RB) {
    float4 q = p[i];
    v[0] += q.x;
    v[1] += q.y;
    v[2] += q.z;
  }
  block_sum<3>(v);
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; ++k) part[3 * blockIdx.x + k] = v[k];
}

__global__ void k_mean3(const double* __restrict__ part, int g, int64_t n, double* out) {
  double v[3] = {0, 0, 0};
  for (int b = threadIdx.x; b < g; b += RB)
    for (int k = 0; k < 3; ++k) v[k] += part[3 * b + k];
  block_sum<3>(v);
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; ++k) out[k] = v[k] / (double)n;
}

int centroid4(const float4* p, int64_t n, double* d_out3, cudaStream_t s) {
  const int g = red_grid(n);
  double* part = nullptr;
  int rc = dev_alloc_n(&part, (size_t)3 * g, s);
  if (rc) return rc;
  k_sum4<<<g, RB, 0, s>>>(p, n, part);
  FGA_LAUNCH_CHECK("sum4");
  k_mean3<<<1, RB, 0, s>>>(part, g, n, d_out3);
  FGA_LAUNCH_CHECK("mean3");
  dev_free(part, s);
  return FGA_OK;
}

}  // namespace fga
