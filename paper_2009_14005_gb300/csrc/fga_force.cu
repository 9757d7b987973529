// Per-iteration kernels of Algorithm 2's loop body:
//   k_direct    all-pairs gravitational force, Eq. 6 (tiled, FP32, rsqrt on MUFU)
//   k_bh        BHForce with the opening criterion of Eq. 15 (warp-cooperative)
//   k_epilogue  Eqs. 7-10 (velocity, displacement), FP64 reductions and, in the
//               last block to finish, the rigid fit of Eqs. 14 and 16 plus the
//               composition R = R'R, t = R't + t' and the convergence test.
// The template is placed on the fly as y = R y0 + t from the accumulated
// transform, so it never drifts from repeated FP32 updates.
#include <algorithm>
#include <atomic>
#include <cmath>

#include "fga_device.cuh"
#include "fga_epi.cuh"

namespace fga {

// ------------------------------------------------------------------ Eq. 6, all pairs
//
// Block of BS threads, each thread owns QPT template points. Sources are
// staged through shared memory one tile of BS sources at a time; every thread
// reads the same source (a broadcast). Per pair: 3 FADD, 3 FFMA
// (r^2 + eps^2), one MUFU rsqrt, 3 FMUL (m / r^3), 3 FFMA (accumulate); with
// an even QPT the thread's points go in pairs through the packed two-wide
// FP32 instructions (pair_term2), half the issue slots for the same results.
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
  // even QPT: template points in pairs, each source staged as (x, x, y, y),
  // (z, z, m, m) so that the packed FP32 instructions serve both points
  constexpr bool PAIRED = QPT % 2 == 0;
  __shared__ float4 tile[PAIRED ? 2 * BS : BS];
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
    const float4 src = j < j1 ? X[j] : make_float4(0.f, 0.f, 0.f, 0.f);  // m = 0 pads the tail
    if constexpr (PAIRED) {
      tile[2 * threadIdx.x] = make_float4(src.x, src.x, src.y, src.y);
      tile[2 * threadIdx.x + 1] = make_float4(src.z, src.z, src.w, src.w);
    } else {
      tile[threadIdx.x] = src;
    }
    __syncthreads();
    float px[QPT], py[QPT], pz[QPT];
    if constexpr (PAIRED) {
      constexpr int NPR = QPT / 2;
      f2 ax[NPR], ay[NPR], az[NPR], nyx[NPR], nyy[NPR], nyz[NPR];
      const f2 e2 = f2_pack(eps2, eps2);
#pragma unroll
      for (int r = 0; r < NPR; ++r) {
        ax[r] = ay[r] = az[r] = f2_pack(0.f, 0.f);
        nyx[r] = f2_pack(-yx[2 * r], -yx[2 * r + 1]);
        nyy[r] = f2_pack(-yy[2 * r], -yy[2 * r + 1]);
        nyz[r] = f2_pack(-yz[2 * r], -yz[2 * r + 1]);
      }
#pragma unroll 8
      for (int k = 0; k < BS; ++k) {
        const float4 sxy = tile[2 * k], szm = tile[2 * k + 1];
#pragma unroll
        for (int r = 0; r < NPR; ++r) pair_term2(sxy, szm, nyx[r], nyy[r], nyz[r], e2, ax[r], ay[r], az[r]);
      }
#pragma unroll
      for (int r = 0; r < NPR; ++r) {
        f2_unpack(ax[r], px[2 * r], px[2 * r + 1]);
        f2_unpack(ay[r], py[2 * r], py[2 * r + 1]);
        f2_unpack(az[r], pz[2 * r], pz[2 * r + 1]);
      }
    } else {
#pragma unroll
      for (int q = 0; q < QPT; ++q) px[q] = py[q] = pz[q] = 0.f;
#pragma unroll 8
      for (int k = 0; k < BS; ++k) {
        const float4 s = tile[k];
#pragma unroll
        for (int q = 0; q < QPT; ++q) {
          const float dx = s.x - yx[q], dy = s.y - yy[q], dz = s.z - yz[q];
          const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
          const float inv = rsqrt_fast(r2);
          const float w = s.w * (inv * inv * inv);
          px[q] = fmaf(w, dx, px[q]);
          py[q] = fmaf(w, dy, py[q]);
          pz[q] = fmaf(w, dz, pz[q]);
        }
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

// Tile shape (threads per block, template points per thread) per template
// size class: M < 8k, M < 64k, M >= 64k. Encoded bs * 16 + qpt; the
// autotuner may replace the defaults.
static std::atomic<int> g_direct_tile[3] = {{128 * 16 + 2}, {256 * 16 + 1}, {256 * 16 + 2}};

int direct_size_class(int64_t M) { return M < 8 * 1024 ? 0 : (M < 64 * 1024 ? 1 : 2); }

bool direct_tile_supported(int bs, int qpt) {
  return (bs == 128 || bs == 256) && (qpt == 1 || qpt == 2 || qpt == 4);
}

void set_direct_tile(int size_class, int bs, int qpt) {
  if (size_class >= 0 && size_class < 3 && direct_tile_supported(bs, qpt))
    g_direct_tile[size_class].store(bs * 16 + qpt);
}

void get_direct_tile(int size_class, int* bs, int* qpt) {
  const int v = g_direct_tile[size_class].load();
  *bs = v / 16;
  *qpt = v % 16;
}

DirectPlan plan_direct(int64_t N, int64_t M) {
  DirectPlan p;
  const int64_t sms = sm_count();
  get_direct_tile(direct_size_class(M), &p.bs, &p.qpt);
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
#define FGA_DIRECT_CASE(B, Q)                                                               \
  else if (plan.bs == B && plan.qpt == Q)                                                   \
    k_direct<B, Q><<<grid, B, 0, s>>>(X, N, plan.chunk, Y0, M, ds, eps2, fb.hi, fb.lo);
  if (false) {
  }
  FGA_DIRECT_CASE(128, 1)
  FGA_DIRECT_CASE(128, 2)
  FGA_DIRECT_CASE(128, 4)
  FGA_DIRECT_CASE(256, 1)
  FGA_DIRECT_CASE(256, 2)
  FGA_DIRECT_CASE(256, 4)
#undef FGA_DIRECT_CASE
  else {
    set_error("launch_direct: unsupported tile shape");
    return FGA_EINTERNAL;
  }
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
// The tree is read as depth-first records (fga_tree::node_pre): CoM + mass
// (16 bytes) and l^2 + subtree record count (8 bytes) in separate arrays, so
// a 128-byte line holds 8 and 16 consecutive records. A walk needs no
// stack: after a record whose cell the point accepts it skips the subtree,
// after a rejected one it continues with the next record (the first child).
// Warps hold 32 Morton-neighbouring points, so their walks touch mostly the
// same records and the loads are served by L1.
//
// Work is split into tasks (group of template points, frontier cell): a task
// first judges the frontier cell's ancestors (a point accepting one stops;
// the monopole is added by the task owning the ancestor's first frontier
// cell), then walks the frontier cell's subtree. Two walks: per lane (32-point
// groups, bh_task_pre) or cooperative (64-point groups, one walk for the
// warp, bh_walk<2>), chosen by bh_walk_kind. Tasks are handed out
// dynamically from a counter in DevState; the last warp to finish resets it.
static constexpr int BH_WARPS = FGA_BH_WARPS;

#ifndef FGA_BH_MINBLOCKS
#define FGA_BH_MINBLOCKS 9  // resident blocks per SM the register budget is sized for
#endif
// KIND (bh_walk_kind): 0 = one template point per lane, each lane walking its
// own point over the depth-first records (bh_task_pre); 2 = two points per
// lane, one walk for the warp with saved sibling ranges (bh_walk); 3 / 4 =
// two / one points per lane, one walk for the warp that follows every
// point's own walk (bh_walk_cursor).
// Resident blocks per SM the register budget of each walk is sized for: 36
// warps per SM at 56 registers (the union walk on planar 1M: 4.88 ms per
// launch, against 5.39 ms with 32 warps at 64 registers and 5.45 ms with 40
// warps at 48; the per-lane walk on LiDAR 120k: 0.658 against 0.667 ms); the
// walk with four points per lane holds twice the per-point registers.
constexpr int bh_min_blocks(int kind) { return kind == 5 ? FGA_BH_MINBLOCKS / 2 : FGA_BH_MINBLOCKS; }

template <int KIND>
__global__ void __launch_bounds__(BH_WARPS * 32, bh_min_blocks(KIND)) k_bh(const float4* __restrict__ pcm,
                                                         const float2* __restrict__ pls,
                                                         const int2* __restrict__ pcf,
                                                         const float4* __restrict__ Y0, int64_t M,
                                                         const FrontCell* __restrict__ front, int K,
                                                         int C,
                                                         DevState* __restrict__ ds, float eps2,
                                                         float theta2, long long* __restrict__ acc,
                                                         float acc_scale,
                                                         const unsigned* __restrict__ order,
                                                         unsigned* __restrict__ cost,
                                                         unsigned* __restrict__ terms) {
  constexpr int PL = (KIND == 0 || KIND == 4) ? 1 : (KIND == 5 ? 4 : 2);  // template points per lane
  if (ds->done) return;
  const int lane = threadIdx.x & 31;
  const Xf xf = load_xf(ds);
  const unsigned ntasks = bh_tasks(M, C, PL);
  unsigned long long total = 0;
#if FGA_BH_BLOCK_TASKS
  __shared__ unsigned s_slot;
#endif
  for (;;) {
    unsigned slot = 0;
#if FGA_BH_BLOCK_TASKS
    if (threadIdx.x == 0) s_slot = atomicAdd(&ds->bh_next, 1u);
    __syncthreads();
    slot = s_slot;
    __syncthreads();
#else
    if (lane == 0) slot = atomicAdd(&ds->bh_next, 1u);
    slot = __shfl_sync(FULL, slot, 0);
#endif
    if (slot >= ntasks) break;
    unsigned task = order ? order[slot] : slot;
    if (task >= ntasks) task = slot;  // never index past the task range
#if FGA_BH_BLOCK_TASKS
    // the block's warps take adjacent groups; a group past the template has
    // no valid point and adds nothing
    const unsigned g = (task / (unsigned)C) * BH_WARPS + (threadIdx.x >> 5), c = task % (unsigned)C;
#else
    const unsigned g = task / (unsigned)C, c = task % (unsigned)C;
#endif
    const unsigned f0 = (unsigned)(((uint64_t)c * K) / C), f1 = (unsigned)(((uint64_t)(c + 1) * K) / C);
    int64_t i[PL];
    bool valid[PL];
    float3 y[PL];
    float h[PL][3], lo[PL][3];
    unsigned cnt[PL];
#pragma unroll
    for (int q = 0; q < PL; ++q) {
      i[q] = (int64_t)g * (32 * PL) + 32 * q + lane;
      valid[q] = i[q] < M;
      y[q] = place(xf, Y0[valid[q] ? i[q] : 0]);
      h[q][0] = h[q][1] = h[q][2] = lo[q][0] = lo[q][1] = lo[q][2] = 0.f;
      cnt[q] = 0u;
    }
    unsigned steps = 0;
    for (unsigned f = f0; f < f1; ++f) {
      if constexpr (KIND == 0)
        bh_task_pre(pcm, pls, front, f, y[0], valid[0], eps2, theta2, h[0][0], h[0][1], h[0][2],
                    lo[0][0], lo[0][1], lo[0][2], cnt[0], steps);
      else if constexpr (KIND == 2)
        bh_walk<2>(pcm, pls, pcf, front, f, y, valid, eps2, theta2, h, lo, cnt, steps);
      else
        bh_walk_cursor<PL>(pcm, pls, front, f, y, valid, eps2, theta2, h, lo, cnt, steps);
    }
    if (cost && lane == 0 && (!FGA_BH_BLOCK_TASKS || threadIdx.x == 0)) cost[task] = steps + 1u;
#pragma unroll
    for (int q = 0; q < PL; ++q) {
      // the task's compensated sums join the point's exact fixed-point sums
      // (a point that added no term adds nothing)
      if (valid[q] && cnt[q]) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const long long v = fixed_point(h[q][k], acc_scale) + fixed_point(lo[q][k], acc_scale);
          atomicAdd(reinterpret_cast<unsigned long long*>(&acc[(int64_t)k * M + i[q]]),
                    (unsigned long long)v);
        }
        if (terms) atomicAdd(&terms[i[q]], cnt[q]);
      }
      total += valid[q] ? cnt[q] : 0u;
    }
  }
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

template <int KIND>
static int bh_grid(int64_t M, int C) {
  static std::atomic<int> cached{0};
  int per_sm = cached.load();
  if (per_sm == 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_bh<KIND>, BH_WARPS * 32, 0) != cudaSuccess || b < 1) {
      cudaGetLastError();
      b = 1;
    }
    per_sm = b;
    cached.store(b);
  }
  const int64_t tasks = bh_tasks(M, C, bh_points_per_lane(KIND));
  const int64_t need = FGA_BH_BLOCK_TASKS ? tasks : (tasks + BH_WARPS - 1) / BH_WARPS;
  return (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)per_sm * sm_count()));
}

int bh_walk_kind(int64_t M, int walk) {
  if (walk == FGA_WALK_LANE) return 0;
  if (walk == FGA_WALK_COOP) return 2;
  if (walk == FGA_WALK_CURSOR) return 3;
  if (walk == FGA_WALK_CURSOR32) return 4;
  if (walk == FGA_WALK_CURSOR128) return 5;
  const int64_t warps = (int64_t)sm_count() * 32;
  return M >= (int64_t)FGA_BH_COOP_POINTS_PER_WARP * warps ? 3 : 0;
}

int bh_chunks(int64_t M, int K, int kind) {
  if (FGA_BH_TASKS_PER_WARP <= 0 || K <= 1) return K < 1 ? 1 : K;
  const int pl = bh_points_per_lane(kind);
  const int64_t groups = (M + 32 * pl - 1) / (32 * pl);
  const int64_t target = (int64_t)FGA_BH_TASKS_PER_WARP * sm_count() * BH_WARPS * bh_min_blocks(kind);
  const int64_t c = (target + groups - 1) / groups;
  return (int)std::max<int64_t>(1, std::min<int64_t>(c, K));
}

int launch_bh(const fga_tree* t, const float4* Y0, int64_t M, DevState* ds, float eps,
              float theta, ForceBuffers& fb, cudaStream_t s, int kind, const unsigned* order, unsigned* cost,
              unsigned* terms) {
  if (!fb.acc) {
    set_error("launch_bh: no fixed-point sums");
    return FGA_EINTERNAL;
  }
  const int C = bh_chunks(M, t->n_front, kind);
  fb.acc_exp = fixed_point_exponent(t->mass_total, eps);
  const float scale = ldexpf(1.0f, fb.acc_exp);
#define FGA_BH_CASE(KD)                                                                           \
  k_bh<KD><<<bh_grid<KD>(M, C), BH_WARPS * 32, 0, s>>>(pre_cm(t), pre_ls(t), pre_cf(t), Y0, M,      \
                                                       t->front, t->n_front, C,                     \
                                                       ds, eps * eps, theta * theta, fb.acc, scale, \
                                                       order, cost, terms)
  if (kind == 2)
    FGA_BH_CASE(2);
  else if (kind == 3)
    FGA_BH_CASE(3);
  else if (kind == 4)
    FGA_BH_CASE(4);
  else if (kind == 5)
    FGA_BH_CASE(5);
  else
    FGA_BH_CASE(0);
#undef FGA_BH_CASE
  FGA_LAUNCH_CHECK("bh");
  return FGA_OK;
}

int fixed_point_exponent(double mass_total, float eps) {
  const double bound = mass_total / (2.598 * (double)eps * (double)eps);
  if (!(bound > 0.0) || !std::isfinite(bound)) return 100;
  int e = 0;
  std::frexp(bound, &e);  // bound < 2^e
  return std::max(-100, std::min(100, 61 - e));
}

// ------------------------------------------------------------------ heavy-first task order
// Counting sort of task indices by descending floor(log2(cost)) over 32
// buckets (bucket = clz(cost), heavier first), in three launches: per-block
// bucket counts, their exclusive scan (bucket-major, so bucket 0 of every
// block precedes bucket 1 of any block), and the scatter. The order within a
// bucket is arbitrary; a task's result never depends on when it runs.
constexpr int ORD_BS = 256;

__device__ __forceinline__ unsigned cost_bucket(const unsigned* __restrict__ cost, unsigned t, unsigned n) {
  return t < n ? (unsigned)__clz(cost[t] | 1u) : 32u;
}

__global__ void __launch_bounds__(ORD_BS) k_ord_hist(const unsigned* __restrict__ cost, unsigned n, unsigned per,
                                                     unsigned* __restrict__ hist) {
  __shared__ unsigned h[32];
  if (threadIdx.x < 32) h[threadIdx.x] = 0u;
  __syncthreads();
  const unsigned lane = threadIdx.x & 31u;
  const unsigned t0 = blockIdx.x * per, t1 = min(n, t0 + per);
  for (unsigned base = t0; base < t1; base += ORD_BS) {
    const unsigned t = base + threadIdx.x;
    const unsigned b = t < t1 ? cost_bucket(cost, t, n) : 32u;
    const unsigned peers = __match_any_sync(FULL, b);
    if (b < 32u && lane == (unsigned)(__ffs(peers) - 1)) atomicAdd(&h[b], (unsigned)__popc(peers));
  }
  __syncthreads();
  if (threadIdx.x < 32) hist[threadIdx.x * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of `count` (<= TASK_ORDER_SCRATCH) values in place, one block.
__global__ void __launch_bounds__(1024) k_ord_scan(unsigned* __restrict__ v, unsigned count) {
  __shared__ unsigned part[1024];
  const unsigned per = (count + 1023u) / 1024u;
  const unsigned s0 = threadIdx.x * per, s1 = min(count, s0 + per);
  unsigned sum = 0;
  for (unsigned k = s0; k < s1; ++k) sum += v[k];
  part[threadIdx.x] = sum;
  __syncthreads();
  for (unsigned off = 1; off < 1024; off <<= 1) {
    const unsigned add = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
    __syncthreads();
    part[threadIdx.x] += add;
    __syncthreads();
  }
  unsigned run = part[threadIdx.x] - sum;  // exclusive prefix of this thread's slice
  for (unsigned k = s0; k < s1; ++k) {
    const unsigned x = v[k];
    v[k] = run;
    run += x;
  }
}

__global__ void __launch_bounds__(ORD_BS) k_ord_scatter(const unsigned* __restrict__ cost, unsigned n, unsigned per,
                                                        const unsigned* __restrict__ offs,
                                                        unsigned* __restrict__ order) {
  __shared__ unsigned base_b[32];
  if (threadIdx.x < 32) base_b[threadIdx.x] = offs[threadIdx.x * gridDim.x + blockIdx.x];
  __syncthreads();
  const unsigned lane = threadIdx.x & 31u;
  const unsigned t0 = blockIdx.x * per, t1 = min(n, t0 + per);
  for (unsigned base = t0; base < t1; base += ORD_BS) {
    const unsigned t = base + threadIdx.x;
    const unsigned b = t < t1 ? cost_bucket(cost, t, n) : 32u;
    const unsigned peers = __match_any_sync(FULL, b);
    const int leader = __ffs(peers) - 1;
    unsigned start = 0;
    if (b < 32u && (int)lane == leader) start = atomicAdd(&base_b[b], (unsigned)__popc(peers));
    start = __shfl_sync(FULL, start, leader);
    if (b < 32u) order[start + (unsigned)__popc(peers & ((1u << lane) - 1u))] = t;
  }
}

int launch_task_order(const unsigned* cost, unsigned ntasks, unsigned* order, cudaStream_t s) {
  if (ntasks == 0) return FGA_OK;
  const unsigned maxb = TASK_ORDER_SCRATCH / 32u;
  unsigned nb = (ntasks + 4095u) / 4096u;
  nb = nb < 1u ? 1u : (nb > maxb ? maxb : nb);
  const unsigned per = (ntasks + nb - 1u) / nb;
  unsigned* hist = order + ntasks;  // TASK_ORDER_SCRATCH entries after the order
  k_ord_hist<<<nb, ORD_BS, 0, s>>>(cost, ntasks, per, hist);
  FGA_LAUNCH_CHECK("order hist");
  k_ord_scan<<<1, 1024, 0, s>>>(hist, 32u * nb);
  FGA_LAUNCH_CHECK("order scan");
  k_ord_scatter<<<nb, ORD_BS, 0, s>>>(cost, ntasks, per, hist, order);
  FGA_LAUNCH_CHECK("order scatter");
  return FGA_OK;
}

// ------------------------------------------------------------------ Eqs. 7-10 + reductions + Eqs. 14/16

int epilogue_blocks(int64_t M) {
  const int64_t g = (M + EPI_BS - 1) / EPI_BS;
  // at most 2 blocks per SM: each block leaves 27 FP64 partials for the last
  // block to add, and FP64 adds are scarce on this GPU
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 2 * (int64_t)sm_count()));
}

// Per template point (grid-stride): the ODE step and reduction terms of
// epi_point; block partials in FP64; the last block to finish sums them and
// runs rigid_step (Eqs. 14, 16 and the composition).
__global__ void __launch_bounds__(EPI_BS) k_epilogue(const float4* __restrict__ Y0, int64_t M,
                                                     const float4* __restrict__ hi,
                                                     const float4* __restrict__ lo, int S,
                                                     float4* __restrict__ V, DevState* ds,
                                                     double* __restrict__ partials,
                                                     unsigned* __restrict__ counter,
                                                     double* __restrict__ traj, EpiParams ep,
                                                     unsigned long long inter_add,
                                                     long long* __restrict__ acc, float acc_unscale) {
  if (ds->done) return;
  __shared__ bool s_last;
  __shared__ double s_red[NRED];
  const EpiCtx c = load_epi(ds);
  float r[NRED];
#pragma unroll
  for (int k = 0; k < NRED; ++k) r[k] = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)EPI_BS + threadIdx.x; i < M; i += (int64_t)gridDim.x * EPI_BS) {
    if (acc)
      epi_point_fixed(i, Y0, acc, acc_unscale, M, V, ep, c, r);
    else
      epi_point(i, Y0, hi, lo, S, M, V, ep, c, r);
  }
  epi_block_partial(r, partials + (int64_t)blockIdx.x * NRED);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  epi_last_reduce(partials, (int)gridDim.x, s_red);
  rigid_step_block(s_red, M, ds, ep, traj, inter_add);
  if (threadIdx.x == 0) {
    *counter = 0u;
    __threadfence();
  }
}

int launch_epilogue(const float4* Y0, int64_t M, const ForceBuffers& fb, float4* V, DevState* ds,
                    double* d_partials, unsigned* d_counter, double* d_traj, const EpiParams& ep,
                    cudaStream_t s, unsigned long long inter_add) {
  k_epilogue<<<epilogue_blocks(M), EPI_BS, 0, s>>>(Y0, M, fb.hi, fb.lo, fb.S, V, ds, d_partials,
                                                   d_counter, d_traj, ep, inter_add, fb.acc,
                                                   ldexpf(1.0f, -fb.acc_exp));
  FGA_LAUNCH_CHECK("epilogue");
  return FGA_OK;
}

// ------------------------------------------------------------------ helpers for fga_forces

// The force on each template point, G (m_Y) times its sum: the compensated
// sum of the S partial sums, or (acc != null) the exact fixed-point sums,
// which are cleared.
__global__ void k_forces_out(const float4* __restrict__ hi, const float4* __restrict__ lo, int S,
                             long long* __restrict__ acc, float acc_unscale,
                             int64_t M, const float4* __restrict__ Y0, int use_mass, float G,
                             const int* __restrict__ perm, float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M;
       i += (int64_t)gridDim.x * blockDim.x) {
    float sx, sy, sz;
    if (acc) {
      sx = __ll2float_rn(acc[i]) * acc_unscale;
      sy = __ll2float_rn(acc[M + i]) * acc_unscale;
      sz = __ll2float_rn(acc[2 * M + i]) * acc_unscale;
      acc[i] = acc[M + i] = acc[2 * M + i] = 0;
    } else {
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
      sx = ahx + alx;
      sy = ahy + aly;
      sz = ahz + alz;
    }
    const float f = use_mass ? G * Y0[i].w : G;
    const int64_t j = perm ? (int64_t)perm[i] : i;
    out[3 * j] = f * sx;
    out[3 * j + 1] = f * sy;
    out[3 * j + 2] = f * sz;
  }
}

int launch_forces_out(const ForceBuffers& fb, int64_t M, const float4* Y0, int use_mass, float G,
                      const int* perm, float* acc_out, cudaStream_t s) {
  const int64_t g = std::max<int64_t>(1, std::min<int64_t>((M + 255) / 256, 8 * (int64_t)sm_count()));
  k_forces_out<<<(unsigned)g, 256, 0, s>>>(fb.hi, fb.lo, fb.S, fb.acc, ldexpf(1.0f, -fb.acc_exp), M, Y0,
                                           use_mass, G, perm, acc_out);
  FGA_LAUNCH_CHECK("forces_out");
  return FGA_OK;
}

__global__ void k_state_init(DevState* ds, const double* __restrict__ mu0) { state_init(ds, mu0, 0); }

int launch_state_init(DevState* ds, const double* d_mu0, cudaStream_t s) {
  k_state_init<<<1, 1, 0, s>>>(ds, d_mu0);
  FGA_LAUNCH_CHECK("state_init");
  return FGA_OK;
}

}  // namespace fga
