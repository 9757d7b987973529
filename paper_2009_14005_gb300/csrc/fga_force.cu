// Per-iteration kernels of Algorithm 2's loop body:
//   k_direct    all-pairs gravitational force, Eq. 6 (tiled, FP32, rsqrt on MUFU)
//   k_bh        BHForce with the opening criterion of Eq. 15 (warp-cooperative)
//   k_epilogue  Eqs. 7-10 (velocity, displacement), FP64 reductions and, in the
//               last block to finish, the rigid fit of Eqs. 14 and 16 plus the
//               composition R = R'R, t = R't + t' and the convergence test.
// The template is placed on the fly as y = R y0 + t from the accumulated
// transform, so it never drifts from repeated FP32 updates.
#include <algorithm>
#include <cmath>

#include "fga_internal.cuh"

namespace fga {

static constexpr unsigned FULL = 0xffffffffu;

// Knuth's TwoSum: s + e == a + b exactly.
__device__ __forceinline__ void comp_add(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bb = s - hi;
  const float e = (hi - (s - bb)) + (x - bb);
  hi = s;
  lo += e;
}

struct Xf {
  float R[9], t[3];
};

__device__ __forceinline__ Xf load_xf(const DevState* __restrict__ ds) {
  Xf x;
#pragma unroll
  for (int k = 0; k < 9; ++k) x.R[k] = ds->Rf[k];
#pragma unroll
  for (int k = 0; k < 3; ++k) x.t[k] = ds->tf[k];
  return x;
}

__device__ __forceinline__ float3 place(const Xf& x, float4 y0) {
  return make_float3(fmaf(x.R[0], y0.x, fmaf(x.R[1], y0.y, fmaf(x.R[2], y0.z, x.t[0]))),
                     fmaf(x.R[3], y0.x, fmaf(x.R[4], y0.y, fmaf(x.R[5], y0.z, x.t[1]))),
                     fmaf(x.R[6], y0.x, fmaf(x.R[7], y0.y, fmaf(x.R[8], y0.z, x.t[2]))));
}

// ------------------------------------------------------------------ Eq. 6, all pairs
//
// Block of BS threads, each thread owns QPT template points. Sources are
// staged through shared memory one tile of BS float4 (x, y, z, m) at a time;
// every thread reads the same source (a broadcast). Per pair: 3 FADD, 3 FFMA
// (r^2 + eps^2), one MUFU rsqrt, 3 FMUL (m / r^3), 3 FFMA (accumulate).
// Each tile's plain FP32 partial is folded into a TwoSum-compensated
// accumulator. blockIdx.y splits the sources into `chunk`-sized ranges whose
// partials the epilogue adds (compensated) in a fixed order.
template <int BS, int QPT>
__global__ void __launch_bounds__(BS) k_direct(const float4* __restrict__ X, int64_t N, int64_t chunk,
                                               const float4* __restrict__ Y0, int64_t M,
                                               const DevState* __restrict__ ds, float eps2,
                                               float4* __restrict__ hi_out,
                                               float4* __restrict__ lo_out) {
  if (ds->done) return;
  __shared__ float4 tile[BS];
  const Xf xf = load_xf(ds);
  const int split = blockIdx.y;
  const int64_t j0 = (int64_t)split * chunk;
  const int64_t j1 = min(N, j0 + chunk);
  float yx[QPT], yy[QPT], yz[QPT];
  float hx[QPT], hy[QPT], hz[QPT], lx[QPT], ly[QPT], lz[QPT];
  const int64_t qbase = (int64_t)blockIdx.x * BS * QPT + threadIdx.x;
#pragma unroll
  for (int q = 0; q < QPT; ++q) {
    const int64_t i = min(qbase + (int64_t)q * BS, M - 1);
    const float3 y = place(xf, Y0[i]);
    yx[q] = y.x;
    yy[q] = y.y;
    yz[q] = y.z;
    hx[q] = hy[q] = hz[q] = lx[q] = ly[q] = lz[q] = 0.f;
  }
  for (int64_t b = j0; b < j1; b += BS) {
    const int64_t j = b + threadIdx.x;
    tile[threadIdx.x] = j < j1 ? X[j] : make_float4(0.f, 0.f, 0.f, 0.f);  // m = 0 pads the tail
    __syncthreads();
    float px[QPT], py[QPT], pz[QPT];
#pragma unroll
    for (int q = 0; q < QPT; ++q) px[q] = py[q] = pz[q] = 0.f;
#pragma unroll 8
    for (int k = 0; k < BS; ++k) {
      const float4 s = tile[k];
#pragma unroll
      for (int q = 0; q < QPT; ++q) {
        const float dx = s.x - yx[q], dy = s.y - yy[q], dz = s.z - yz[q];
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
        const float inv = rsqrtf(r2);
        const float w = s.w * (inv * inv * inv);
        px[q] = fmaf(w, dx, px[q]);
        py[q] = fmaf(w, dy, py[q]);
        pz[q] = fmaf(w, dz, pz[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < QPT; ++q) {
      comp_add(hx[q], lx[q], px[q]);
      comp_add(hy[q], ly[q], py[q]);
      comp_add(hz[q], lz[q], pz[q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < QPT; ++q) {
    const int64_t i = qbase + (int64_t)q * BS;
    if (i < M) {
      hi_out[(int64_t)split * M + i] = make_float4(hx[q], hy[q], hz[q], 0.f);
      lo_out[(int64_t)split * M + i] = make_float4(lx[q], ly[q], lz[q], 0.f);
    }
  }
}

DirectPlan plan_direct(int64_t N, int64_t M) {
  DirectPlan p;
  const int64_t sms = sm_count();
  if (M >= 64 * 1024) {
    p.bs = 256;
    p.qpt = 2;
  } else if (M >= 8 * 1024) {
    p.bs = 256;
    p.qpt = 1;
  } else {
    p.bs = 128;
    p.qpt = 1;
  }
  const int64_t qblocks = (M + (int64_t)p.bs * p.qpt - 1) / ((int64_t)p.bs * p.qpt);
  const int64_t target = 4 * sms;  // blocks to fill every SM a few times
  int64_t S = std::max<int64_t>(1, (target + qblocks - 1) / qblocks);
  const int64_t tiles = (N + p.bs - 1) / p.bs;
  S = std::min<int64_t>(S, std::max<int64_t>(tiles, 1));
  S = std::min<int64_t>(S, 64);
  const int64_t tiles_per = (tiles + S - 1) / S;
  p.chunk = tiles_per * p.bs;
  p.S = (int)((N + p.chunk - 1) / p.chunk);
  if (p.S < 1) p.S = 1;
  return p;
}

int launch_direct(const float4* X, int64_t N, const float4* Y0, int64_t M, const DevState* ds,
                  float eps, const DirectPlan& plan, ForceBuffers& fb, cudaStream_t s) {
  const float eps2 = eps * eps;
  const int64_t qblocks = (M + (int64_t)plan.bs * plan.qpt - 1) / ((int64_t)plan.bs * plan.qpt);
  dim3 grid((unsigned)qblocks, (unsigned)plan.S);
  if (plan.bs == 256 && plan.qpt == 2)
    k_direct<256, 2><<<grid, 256, 0, s>>>(X, N, plan.chunk, Y0, M, ds, eps2, fb.hi, fb.lo);
  else if (plan.bs == 256)
    k_direct<256, 1><<<grid, 256, 0, s>>>(X, N, plan.chunk, Y0, M, ds, eps2, fb.hi, fb.lo);
  else
    k_direct<128, 1><<<grid, 128, 0, s>>>(X, N, plan.chunk, Y0, M, ds, eps2, fb.hi, fb.lo);
  FGA_LAUNCH_CHECK("direct");
  fb.S = plan.S;
  return FGA_OK;
}

// ------------------------------------------------------------------ BHForce, Eq. 15
//
// Every lane walks the tree for its own template point exactly as BHForce of
// Algorithm 2 does, depth first with children in octant order:
//   * a cell with l / |y - CoM| < theta (written l^2 < theta^2 |y - CoM|^2),
//     or a leaf holding one particle, is added as one particle (Eq. 6 with the
//     cell mass at its CoM);
//   * otherwise an internal cell's children are visited next, and a leaf
//     holding several particles adds each of them exactly.
// The pending work of a lane is one range of unvisited siblings per level,
// packed as (first cell << 4 | count) into one word; the current range lives
// in registers and the rest in a per-lane column of shared memory (at most
// one entry per tree level). A cell record is 32 bytes (CoM + mass, then l^2,
// first child / body, child count, depth), fetched with two loads from the
// same sector. Warps hold 32 Morton-neighbouring points, so their walks touch
// mostly the same cells and the loads are served by L1.
//
// Work is split into tasks (32-point group, frontier cell): a task first
// judges the frontier cell's ancestors (a lane accepting one stops; the
// monopole is added by the task owning the ancestor's first frontier cell),
// then walks the frontier cell's subtree. Tasks are handed out dynamically
// from a counter in DevState; the last warp to finish resets it.
static constexpr int BH_WARPS = 4;
static constexpr int BH_DEPTH = 24;  // > 21 tree levels: one pending range per level

__global__ void __launch_bounds__(BH_WARPS * 32, 8) k_bh(const float4* __restrict__ rec,
                                                         const float4* __restrict__ bodies,
                                                         const float4* __restrict__ Y0, int64_t M,
                                                         const FrontCell* __restrict__ front, int K,
                                                         DevState* __restrict__ ds, float eps2,
                                                         float theta2, float4* __restrict__ hi_out,
                                                         float4* __restrict__ lo_out) {
  if (ds->done) return;
  __shared__ unsigned s_stack[BH_WARPS][BH_DEPTH][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned* const stk = &s_stack[w][0][lane];
  const Xf xf = load_xf(ds);
  const unsigned ntasks = (unsigned)((M + 31) / 32) * (unsigned)K;
  unsigned long long total = 0;
  bool overflow = false;
  for (;;) {
    unsigned task = 0;
    if (lane == 0) task = atomicAdd(&ds->bh_next, 1u);
    task = __shfl_sync(FULL, task, 0);
    if (task >= ntasks) break;
    const unsigned g = task / (unsigned)K, f = task % (unsigned)K;
    const int64_t i = (int64_t)g * 32 + lane;
    const bool valid = i < M;
    const float3 y = place(xf, Y0[valid ? i : 0]);
    float hx = 0.f, hy = 0.f, hz = 0.f, lx = 0.f, ly = 0.f, lz = 0.f;
    float px = 0.f, py = 0.f, pz = 0.f;
    unsigned count = 0;
    bool live = valid;
    {
      const int npath = front[f].npath;
      const unsigned first_mask = front[f].first_mask;
      for (int j = 0; j < npath; ++j) {
        const int a = front[f].path[j];
        const float4 cm = rec[2 * a];
        const float l2 = rec[2 * a + 1].x;
        const float dx = cm.x - y.x, dy = cm.y - y.y, dz = cm.z - y.z;
        const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const bool accept = live && l2 < theta2 * d2;
        if ((first_mask >> j) & 1u) {
          const float inv = rsqrtf(d2 + eps2);
          const float wgt = accept ? cm.w * (inv * inv * inv) : 0.f;
          px = fmaf(wgt, dx, px);
          py = fmaf(wgt, dy, py);
          pz = fmaf(wgt, dz, pz);
          count += accept;
        }
        live = live && !accept;
      }
    }
    // per-lane walk of the frontier cell's subtree
    int cur = front[f].node;  // next cell of the current sibling range
    int cnt = live ? 1 : 0;   // cells left in the current range
    int sp = 0;               // saved ranges in shared memory
    int since_flush = 0;
    while (__any_sync(FULL, cnt > 0)) {
      if (cnt > 0) {
        const int v = cur;
        ++cur;
        --cnt;
        const float4 cm = rec[2 * v];
        const float4 ri = rec[2 * v + 1];
        const int nchild = __float_as_int(ri.z);
        const float dx = cm.x - y.x, dy = cm.y - y.y, dz = cm.z - y.z;
        const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const bool accept = nchild == -1 || ri.x < theta2 * d2;
        const float inv = rsqrtf(d2 + eps2);
        const float wgt = accept ? cm.w * (inv * inv * inv) : 0.f;
        px = fmaf(wgt, dx, px);
        py = fmaf(wgt, dy, py);
        pz = fmaf(wgt, dz, pz);
        count += accept;
        // descend into an internal cell that fails the test: save the rest of
        // the current range, continue with the children (branch-free)
        const bool descend = !accept && nchild > 0;
        const bool save = descend && cnt > 0;
        if (save) {
          if (sp < BH_DEPTH) stk[32 * sp] = ((unsigned)cur << 4) | (unsigned)cnt;
          else overflow = true;
        }
        sp += save;
        cur = descend ? __float_as_int(ri.y) : cur;
        cnt = descend ? nchild : cnt;
        if (!accept && nchild < -1) {
          // leaf holding several particles: add each exactly (rare)
          const int b0 = __float_as_int(ri.y), nb = -nchild;
          for (int b = 0; b < nb; ++b) {
            const float4 q = bodies[b0 + b];
            const float ex = q.x - y.x, ey = q.y - y.y, ez = q.z - y.z;
            const float iq = rsqrtf(fmaf(ex, ex, fmaf(ey, ey, fmaf(ez, ez, eps2))));
            const float wq = q.w * (iq * iq * iq);
            px = fmaf(wq, ex, px);
            py = fmaf(wq, ey, py);
            pz = fmaf(wq, ez, pz);
          }
          count += (unsigned)nb;
        }
        // range exhausted: resume the innermost saved range
        const bool pop = cnt == 0 && sp > 0;
        sp -= pop;
        const unsigned e = (pop && sp < BH_DEPTH) ? stk[32 * sp] : 0u;
        cur = pop ? (int)(e >> 4) : cur;
        cnt = pop ? (int)(e & 15u) : cnt;
      }
      if (++since_flush == 32) {
        comp_add(hx, lx, px);
        comp_add(hy, ly, py);
        comp_add(hz, lz, pz);
        px = py = pz = 0.f;
        since_flush = 0;
      }
    }
    comp_add(hx, lx, px);
    comp_add(hy, ly, py);
    comp_add(hz, lz, pz);
    if (valid) {
      hi_out[(int64_t)f * M + i] = make_float4(hx, hy, hz, 0.f);
      lo_out[(int64_t)f * M + i] = make_float4(lx, ly, lz, 0.f);
    }
    total += valid ? count : 0u;
  }
  if (__any_sync(FULL, overflow) && lane == 0) atomicOr(&ds->status, 1);
  for (int off = 16; off > 0; off >>= 1) total += __shfl_down_sync(FULL, total, off);
  if (lane == 0) {
    if (total) atomicAdd(&ds->interactions, total);
    // the last warp out resets the task counter for the next launch
    __threadfence();
    const unsigned out = atomicAdd(&ds->bh_exited, 1u);
    if (out == gridDim.x * BH_WARPS - 1) {
      ds->bh_next = 0u;
      ds->bh_exited = 0u;
      __threadfence();
    }
  }
}

static int bh_grid(int64_t M, int K) {
  static int per_sm = 0;
  if (per_sm == 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_bh, BH_WARPS * 32, 0) != cudaSuccess || b < 1) {
      cudaGetLastError();
      b = 1;
    }
    per_sm = b;
  }
  const int64_t tasks = (M + 31) / 32 * K;
  const int64_t need = (tasks + BH_WARPS - 1) / BH_WARPS;
  return (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)per_sm * sm_count()));
}

int launch_bh(const fga_tree* t, const float4* Y0, int64_t M, DevState* ds, float eps,
              float theta, ForceBuffers& fb, cudaStream_t s) {
  k_bh<<<bh_grid(M, t->n_front), BH_WARPS * 32, 0, s>>>(t->node_rec, t->bodies, Y0, M, t->front,
                                                        t->n_front, ds, eps * eps, theta * theta,
                                                        fb.hi, fb.lo);
  FGA_LAUNCH_CHECK("bh");
  fb.S = t->n_front;
  return FGA_OK;
}

// ------------------------------------------------------------------ Eqs. 7-10 + reductions + Eqs. 14/16
static constexpr int EPI_BS = 256;

int epilogue_blocks(int64_t M) {
  const int64_t g = (M + EPI_BS - 1) / EPI_BS;
  // at most 2 blocks per SM: each block leaves 27 FP64 partials for the last
  // block to add, and FP64 adds are scarce on this GPU
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 2 * (int64_t)sm_count()));
}

// Symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations (FP64):
// A = V diag(w) V^T, eigenvalues sorted descending, eigenvectors in V's columns.
__device__ void eig_sym3(const double A_in[9], double w[3], double V[9]) {
  double A[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    A[k] = A_in[k];
    V[k] = (k % 4 == 0) ? 1.0 : 0.0;
  }
  for (int sweep = 0; sweep < 32; ++sweep) {
    const double off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
    const double dia = A[0] * A[0] + A[4] * A[4] + A[8] * A[8];
    if (!(off > 1e-32 * dia)) break;
    for (int pq = 0; pq < 3; ++pq) {
      const int p = pq == 2 ? 1 : 0;
      const int q = pq == 0 ? 1 : 2;
      const double apq = A[3 * p + q];
      if (apq == 0.0) continue;
      const double app = A[3 * p + p], aqq = A[3 * q + q];
      const double tau = (aqq - app) / (2.0 * apq);
      const double tn = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
      const double c = 1.0 / sqrt(1.0 + tn * tn), sn = tn * c;
      // A <- J^T A J with J the rotation in the (p, q) plane
      for (int k = 0; k < 3; ++k) {
        const double akp = A[3 * k + p], akq = A[3 * k + q];
        A[3 * k + p] = c * akp - sn * akq;
        A[3 * k + q] = sn * akp + c * akq;
      }
      for (int k = 0; k < 3; ++k) {
        const double apk = A[3 * p + k], aqk = A[3 * q + k];
        A[3 * p + k] = c * apk - sn * aqk;
        A[3 * q + k] = sn * apk + c * aqk;
      }
      for (int k = 0; k < 3; ++k) {
        const double vkp = V[3 * k + p], vkq = V[3 * k + q];
        V[3 * k + p] = c * vkp - sn * vkq;
        V[3 * k + q] = sn * vkp + c * vkq;
      }
    }
  }
  w[0] = A[0];
  w[1] = A[4];
  w[2] = A[8];
  // sort descending (3 elements)
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2 - a; ++b)
      if (w[b] < w[b + 1]) {
        const double tw = w[b];
        w[b] = w[b + 1];
        w[b + 1] = tw;
        for (int k = 0; k < 3; ++k) {
          const double tv = V[3 * k + b];
          V[3 * k + b] = V[3 * k + b + 1];
          V[3 * k + b + 1] = tv;
        }
      }
}

// Proper rotation maximising tr(R^T C): with C = sum_k s_k u_k v_k^T,
// R = u1 v1^T + u2 v2^T + (u1 x u2)(v1 x v2)^T, i.e. U diag(1, 1, sgn det(U V^T)) V^T
// of Eq. 14 written with the two leading singular pairs only. The pairs come
// from the eigenvectors of C^T C (v_k) and u_k = C v_k / |C v_k| (u2 made
// orthogonal to u1). Returns false when the second singular value is below
// 1e-7 of the first (rank(C) < 2: no rotation is determined).
__device__ bool rigid_rotation(const double C[9], double R[9]) {
  double B[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      B[3 * r + c] = C[r] * C[c] + C[3 + r] * C[3 + c] + C[6 + r] * C[6 + c];
  double lam[3], V[9];
  eig_sym3(B, lam, V);
  if (!(lam[0] > 0.0) || !(lam[1] > 1e-14 * lam[0])) return false;
  double v1[3] = {V[0], V[3], V[6]}, v2[3] = {V[1], V[4], V[7]};
  double u1[3], u2[3];
  for (int r = 0; r < 3; ++r) {
    u1[r] = C[3 * r] * v1[0] + C[3 * r + 1] * v1[1] + C[3 * r + 2] * v1[2];
    u2[r] = C[3 * r] * v2[0] + C[3 * r + 1] * v2[1] + C[3 * r + 2] * v2[2];
  }
  const double n1 = sqrt(u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]);
  for (int r = 0; r < 3; ++r) u1[r] /= n1;
  const double pr = u1[0] * u2[0] + u1[1] * u2[1] + u1[2] * u2[2];
  for (int r = 0; r < 3; ++r) u2[r] -= pr * u1[r];
  const double n2 = sqrt(u2[0] * u2[0] + u2[1] * u2[1] + u2[2] * u2[2]);
  if (!(n2 > 0.0)) return false;
  for (int r = 0; r < 3; ++r) u2[r] /= n2;
  const double u3[3] = {u1[1] * u2[2] - u1[2] * u2[1], u1[2] * u2[0] - u1[0] * u2[2],
                        u1[0] * u2[1] - u1[1] * u2[0]};
  const double v3[3] = {v1[1] * v2[2] - v1[2] * v2[1], v1[2] * v2[0] - v1[0] * v2[2],
                        v1[0] * v2[1] - v1[1] * v2[0]};
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) R[3 * r + c] = u1[r] * v1[c] + u2[r] * v2[c] + u3[r] * v3[c];
  return true;
}

// FP64 on this GPU has long dependent latencies (about 64 cycles per DFMA and
// over 600 per division or square root), and the rigid fit is one thread's
// dependency chain on the iteration's critical path. So the chain avoids FP64
// division and square root: reciprocals are an FP32 seed refined by two
// Newton steps in FP64 (r <- r + r (1 - d r), 24 -> 48 -> 53 bits), and sums
// are pairwise.
__device__ __forceinline__ double rcp64(double d) {
  double r = (double)__frcp_rn((float)d);
  r = fma(r, fma(-d, r, 1.0), r);
  r = fma(r, fma(-d, r, 1.0), r);
  return r;
}

__device__ __forceinline__ double sum9(const double v[9]) {
  return ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])) + v[8];
}

// Orthogonal polar factor of C by the scaled Newton iteration
// X <- (g X + X^{-T} / g) / 2 (Higham), started from a positive multiple of C.
// For det C > 0 the limit is U V^T of C = U S V^T, i.e. Eq. 14's rotation
// (sgn det(U V^T) = +1). Any g > 0 keeps the same limit, so the scaling
// g = (|X^{-1}|_F / |X|_F)^{1/2} and the start scale are computed in FP32;
// the iterates themselves are FP64. Returns false when C is not safely
// positive-determinant (the caller then takes the eigen-decomposition route,
// which also handles rank deficiency).
__device__ bool polar_rotation(const double C[9], double R[9]) {
  double sq[9];
  for (int k = 0; k < 9; ++k) sq[k] = C[k] * C[k];
  const double nc2 = sum9(sq);
  if (!(nc2 > 0.0) || !isfinite(nc2)) return false;
  const double s0 = (double)rsqrtf((float)nc2);
  double X[9];
  for (int k = 0; k < 9; ++k) X[k] = C[k] * s0;
  bool scaled = true;  // unscaled steps near the limit: an FP32 g would move the fixed point
  for (int it = 0; it < 30; ++it) {
    // cofactors: X^{-T} = cof(X) / det(X)
    double cf[9];
    cf[0] = fma(X[4], X[8], -X[5] * X[7]);
    cf[1] = fma(X[5], X[6], -X[3] * X[8]);
    cf[2] = fma(X[3], X[7], -X[4] * X[6]);
    cf[3] = fma(X[2], X[7], -X[1] * X[8]);
    cf[4] = fma(X[0], X[8], -X[2] * X[6]);
    cf[5] = fma(X[1], X[6], -X[0] * X[7]);
    cf[6] = fma(X[1], X[5], -X[2] * X[4]);
    cf[7] = fma(X[2], X[3], -X[0] * X[5]);
    cf[8] = fma(X[0], X[4], -X[1] * X[3]);
    const double det = fma(X[0], cf[0], fma(X[1], cf[1], X[2] * cf[2]));
    if (!(det > 1e-9)) return false;  // |X|_F ~ 1: a small det means near rank 2
    const double idet = rcp64(det);
    double xx[9], ii[9];
    for (int k = 0; k < 9; ++k) {
      cf[k] *= idet;
      xx[k] = X[k] * X[k];
      ii[k] = cf[k] * cf[k];
    }
    const float g = scaled ? sqrtf(sqrtf((float)sum9(ii) / (float)sum9(xx))) : 1.0f;
    const double a = 0.5 * (double)g, b = 0.5 * (double)(1.0f / g);
    double dd[9];
    for (int k = 0; k < 9; ++k) {
      const double xn = fma(a, X[k], b * cf[k]);
      dd[k] = (xn - X[k]) * (xn - X[k]);
      X[k] = xn;
    }
    const double change = sum9(dd);
    if (!scaled && change < 1e-28) break;
    if (change < 1e-8) scaled = false;
  }
  for (int k = 0; k < 9; ++k) R[k] = X[k];
  return true;
}

// One thread: reductions -> C -> (R', t') -> compose, convergence, next-iteration constants.
__device__ void rigid_step(const double* red, int64_t M, DevState* ds, const EpiParams& ep,
                           double* traj, unsigned long long inter_add) {
  const double Md = (double)M;
  double ybar[3], mud[3];
  for (int k = 0; k < 3; ++k) {
    ybar[k] = red[k] * ep.inv_M;     // mean of the centred template (~0)
    mud[k] = red[3 + k] * ep.inv_M;  // mean displacement
  }
  // symmetric S = sum yc yc^T (xx, xy, xz, yy, yz, zz) and Dy = sum d yc^T
  const double S[9] = {red[6], red[7], red[8], red[7], red[9], red[10], red[8], red[10], red[11]};
  double C[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      C[3 * r + c] = S[3 * r + c] + red[12 + 3 * r + c] - Md * (ybar[r] + mud[r]) * ybar[c];
  double Rp[9];
  const bool ok = polar_rotation(C, Rp) || rigid_rotation(C, Rp);
  if (!ok) {
    for (int k = 0; k < 9; ++k) Rp[k] = (k % 4 == 0) ? 1.0 : 0.0;
    ds->degenerate += 1;
  }
  // mu_Y = muf + ybar (muf is the FP32 centre the kernels subtracted)
  double muy[3];
  for (int k = 0; k < 3; ++k) muy[k] = (double)ds->muf[k] + ybar[k];
  double tp[3];
  for (int r = 0; r < 3; ++r)
    tp[r] = muy[r] + mud[r] - (Rp[3 * r] * muy[0] + Rp[3 * r + 1] * muy[1] + Rp[3 * r + 2] * muy[2]);
  double Rn[9], tn[3];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c)
      Rn[3 * r + c] = Rp[3 * r] * ds->R[c] + Rp[3 * r + 1] * ds->R[3 + c] + Rp[3 * r + 2] * ds->R[6 + c];
    tn[r] = Rp[3 * r] * ds->t[0] + Rp[3 * r + 1] * ds->t[1] + Rp[3 * r + 2] * ds->t[2] + tp[r];
  }
  double T[12];
  for (int k = 0; k < 9; ++k) T[k] = Rn[k];
  for (int k = 0; k < 3; ++k) T[9 + k] = tn[k];
  const int k_it = ds->iter;
  if (k_it >= 2) {
    double d2 = 0;
    for (int q = 0; q < 12; ++q) d2 += (T[q] - ds->Tm2[q]) * (T[q] - ds->Tm2[q]);
    ds->last_conv = d2;
    if (ep.conv_tol > 0 && d2 <= ep.conv_tol) ds->done = 1;
  } else {
    ds->last_conv = -1.0;
  }
  for (int q = 0; q < 12; ++q) {
    ds->Tm2[q] = ds->Tm1[q];
    ds->Tm1[q] = T[q];
  }
  bool finite = true;
  for (int q = 0; q < 12; ++q) finite = finite && isfinite(T[q]);
  if (!finite) {
    ds->status |= 2;
    ds->done = 1;
  }
  for (int k = 0; k < 9; ++k) {
    ds->R[k] = Rn[k];
    ds->Rf[k] = (float)Rn[k];
  }
  for (int k = 0; k < 3; ++k) {
    ds->t[k] = tn[k];
    ds->tf[k] = (float)tn[k];
  }
  for (int r = 0; r < 3; ++r)
    ds->muf[r] = (float)(Rn[3 * r] * ds->mu0[0] + Rn[3 * r + 1] * ds->mu0[1] +
                         Rn[3 * r + 2] * ds->mu0[2] + tn[r]);
  // rigid velocity of the next iteration: v = (y_new - y_old)/dt with
  // y_old = R'^T (y_new - t'), i.e. v = (I - R'^T)/dt y_new + R'^T t'/dt
  const double idt = ep.inv_dt;
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c)
      ds->A[3 * r + c] = (float)(((r == c ? 1.0 : 0.0) - Rp[3 * c + r]) * idt);
    ds->b[r] = (float)((Rp[r] * tp[0] + Rp[3 + r] * tp[1] + Rp[6 + r] * tp[2]) * idt);
  }
  for (int k = 0; k < 3; ++k) {
    ds->netF[k] = red[21 + k];
    ds->torque[k] = red[24 + k];
  }
  if (traj && k_it < ep.max_traj)
    for (int q = 0; q < 12; ++q) traj[12 * (int64_t)k_it + q] = T[q];
  ds->interactions += inter_add;
  ds->iter = k_it + 1;
}

// Per template point (grid-stride): a = G * force sum; Eq. 9 with the
// dissipative force of Eq. 7, v' = v + dt (a - eta v / m_Y); Eq. 10, d = dt v'.
// Per-thread and per-warp sums are FP32 (a few dozen terms); everything above
// the warp is FP64 in a fixed order. The last block to finish reduces the
// per-block partials and runs rigid_step.
__global__ void __launch_bounds__(EPI_BS) k_epilogue(const float4* __restrict__ Y0, int64_t M,
                                                     const float4* __restrict__ hi,
                                                     const float4* __restrict__ lo, int S,
                                                     float4* __restrict__ V, DevState* ds,
                                                     double* __restrict__ partials,
                                                     unsigned* __restrict__ counter,
                                                     double* __restrict__ traj, EpiParams ep,
                                                     unsigned long long inter_add) {
  if (ds->done) return;
  __shared__ double s_w[EPI_BS / 32][NRED];
  __shared__ bool s_last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const Xf xf = load_xf(ds);
  const float mu0 = ds->muf[0], mu1 = ds->muf[1], mu2 = ds->muf[2];
  float A[9], bb[3];
#pragma unroll
  for (int k = 0; k < 9; ++k) A[k] = ds->A[k];
#pragma unroll
  for (int k = 0; k < 3; ++k) bb[k] = ds->b[k];
  float r[NRED];
#pragma unroll
  for (int k = 0; k < NRED; ++k) r[k] = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)EPI_BS + threadIdx.x; i < M; i += (int64_t)gridDim.x * EPI_BS) {
    const float4 y0 = Y0[i];
    const float3 y = place(xf, y0);
    const float cx = y.x - mu0, cy = y.y - mu1, cz = y.z - mu2;
    float ahx = 0.f, ahy = 0.f, ahz = 0.f, alx = 0.f, aly = 0.f, alz = 0.f;
    for (int s = 0; s < S; s += 4) {
      // four independent loads in flight, then the same in-order compensated sum
      float4 h[4], l[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const bool ok = s + k < S;
        h[k] = ok ? hi[(int64_t)(s + k) * M + i] : make_float4(0.f, 0.f, 0.f, 0.f);
        l[k] = ok ? lo[(int64_t)(s + k) * M + i] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        comp_add(ahx, alx, h[k].x);
        comp_add(ahy, aly, h[k].y);
        comp_add(ahz, alz, h[k].z);
        alx += l[k].x;
        aly += l[k].y;
        alz += l[k].z;
      }
    }
    const float ax = ep.G * (ahx + alx), ay = ep.G * (ahy + aly), az = ep.G * (ahz + alz);
    float vx, vy, vz;
    if (ep.vmode == FGA_VEL_RIGID) {
      vx = fmaf(A[0], y.x, fmaf(A[1], y.y, fmaf(A[2], y.z, bb[0])));
      vy = fmaf(A[3], y.x, fmaf(A[4], y.y, fmaf(A[5], y.z, bb[1])));
      vz = fmaf(A[6], y.x, fmaf(A[7], y.y, fmaf(A[8], y.z, bb[2])));
    } else {
      const float4 v = V[i];
      vx = v.x;
      vy = v.y;
      vz = v.z;
    }
    const float kd = ep.eta / y0.w;
    vx = vx + ep.dt * (ax - kd * vx);
    vy = vy + ep.dt * (ay - kd * vy);
    vz = vz + ep.dt * (az - kd * vz);
    if (ep.vmode != FGA_VEL_RIGID) V[i] = make_float4(vx, vy, vz, 0.f);
    const float dx = ep.dt * vx, dy = ep.dt * vy, dz = ep.dt * vz;
    const float fx = y0.w * ax, fy = y0.w * ay, fz = y0.w * az;
    r[0] += cx; r[1] += cy; r[2] += cz;
    r[3] += dx; r[4] += dy; r[5] += dz;
    r[6] += cx * cx; r[7] += cx * cy; r[8] += cx * cz;
    r[9] += cy * cy; r[10] += cy * cz; r[11] += cz * cz;
    r[12] += dx * cx; r[13] += dx * cy; r[14] += dx * cz;
    r[15] += dy * cx; r[16] += dy * cy; r[17] += dy * cz;
    r[18] += dz * cx; r[19] += dz * cy; r[20] += dz * cz;
    r[21] += fx; r[22] += fy; r[23] += fz;
    r[24] += cy * fz - cz * fy;
    r[25] += cz * fx - cx * fz;
    r[26] += cx * fy - cy * fx;
  }
#pragma unroll
  for (int k = 0; k < NRED; ++k)
    for (int off = 16; off > 0; off >>= 1) r[k] += __shfl_down_sync(FULL, r[k], off);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NRED; ++k) s_w[w][k] = (double)r[k];
  __syncthreads();
  if (threadIdx.x < NRED) {
    double acc = 0;
    for (int ww = 0; ww < EPI_BS / 32; ++ww) acc += s_w[ww][threadIdx.x];
    partials[(int64_t)blockIdx.x * NRED + threadIdx.x] = acc;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // last block: FP64 sum over the per-block partials in a fixed order.
  // Thread t < 8 * NRED adds value k = t % NRED over blocks j, j + 8, ...
  // (j = t / NRED); then NRED threads add the 8 strands.
  __shared__ double s_strand[8][NRED];
  __shared__ double s_red[NRED];
  if (threadIdx.x < 8 * NRED) {
    const int k = threadIdx.x % NRED, j = threadIdx.x / NRED;
    double acc = 0.0;
    for (int b = j; b < (int)gridDim.x; b += 8) acc += __ldcg(&partials[(int64_t)b * NRED + k]);
    s_strand[j][k] = acc;
  }
  __syncthreads();
  if (threadIdx.x < NRED) {
    double acc = 0.0;
    for (int j = 0; j < 8; ++j) acc += s_strand[j][threadIdx.x];
    s_red[threadIdx.x] = acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double red[NRED];
    for (int k = 0; k < NRED; ++k) red[k] = s_red[k];
    rigid_step(red, M, ds, ep, traj, inter_add);
    *counter = 0u;
    __threadfence();
  }
}

int launch_epilogue(const float4* Y0, int64_t M, const ForceBuffers& fb, float4* V, DevState* ds,
                    double* d_partials, unsigned* d_counter, double* d_traj, const EpiParams& ep,
                    cudaStream_t s, unsigned long long inter_add) {
  k_epilogue<<<epilogue_blocks(M), EPI_BS, 0, s>>>(Y0, M, fb.hi, fb.lo, fb.S, V, ds, d_partials,
                                                   d_counter, d_traj, ep, inter_add);
  FGA_LAUNCH_CHECK("epilogue");
  return FGA_OK;
}

// ------------------------------------------------------------------ helpers for fga_forces

__global__ void k_forces_out(const float4* __restrict__ hi, const float4* __restrict__ lo, int S,
                             int64_t M, const float4* __restrict__ Y0, int use_mass, float G,
                             const int* __restrict__ perm, float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M;
       i += (int64_t)gridDim.x * blockDim.x) {
    float ahx = 0.f, ahy = 0.f, ahz = 0.f, alx = 0.f, aly = 0.f, alz = 0.f;
    for (int s = 0; s < S; ++s) {
      const float4 h = hi[(int64_t)s * M + i];
      const float4 l = lo[(int64_t)s * M + i];
      comp_add(ahx, alx, h.x);
      comp_add(ahy, aly, h.y);
      comp_add(ahz, alz, h.z);
      alx += l.x;
      aly += l.y;
      alz += l.z;
    }
    const float f = use_mass ? G * Y0[i].w : G;
    const int64_t j = perm ? (int64_t)perm[i] : i;
    out[3 * j] = f * (ahx + alx);
    out[3 * j + 1] = f * (ahy + aly);
    out[3 * j + 2] = f * (ahz + alz);
  }
}

int launch_forces_out(const ForceBuffers& fb, int64_t M, const float4* Y0, int use_mass, float G,
                      const int* perm, float* acc_out, cudaStream_t s) {
  const int64_t g = std::max<int64_t>(1, std::min<int64_t>((M + 255) / 256, 8 * (int64_t)sm_count()));
  k_forces_out<<<(unsigned)g, 256, 0, s>>>(fb.hi, fb.lo, fb.S, M, Y0, use_mass, G, perm, acc_out);
  FGA_LAUNCH_CHECK("forces_out");
  return FGA_OK;
}

__global__ void k_state_init(DevState* ds, const double* __restrict__ mu0) {
  DevState z;
  for (int k = 0; k < 9; ++k) {
    z.R[k] = (k % 4 == 0) ? 1.0 : 0.0;
    z.Rf[k] = (float)z.R[k];
    z.A[k] = 0.f;
  }
  for (int k = 0; k < 12; ++k) z.Tm1[k] = z.Tm2[k] = (k < 9 && k % 4 == 0) ? 1.0 : 0.0;
  for (int k = 0; k < 3; ++k) {
    z.t[k] = 0.0;
    z.tf[k] = 0.f;
    z.b[k] = 0.f;
    z.mu0[k] = mu0 ? mu0[k] : 0.0;
    z.muf[k] = (float)z.mu0[k];
    z.netF[k] = z.torque[k] = 0.0;
  }
  z.last_conv = -1.0;
  z.interactions = 0ull;
  z.iter = 0;
  z.done = 0;
  z.status = 0;
  z.degenerate = 0;
  z.bh_next = 0u;
  z.bh_exited = 0u;
  *ds = z;
}

int launch_state_init(DevState* ds, const double* d_mu0, cudaStream_t s) {
  k_state_init<<<1, 1, 0, s>>>(ds, d_mu0);
  FGA_LAUNCH_CHECK("state_init");
  return FGA_OK;
}

}  // namespace fga
