// Batched registration: many independent pairs of uneven size advance
// together, one iteration of Algorithm 2 for all of them per pair of launches,
// and the whole loop is captured in one CUDA graph.
//
// Force launch: the warp tasks of all pairs are numbered consecutively, pair
// by pair (a prefix sum over the pairs maps a task to its pair by binary
// search); warps take tasks from a device counter. A Barnes-Hut task is (pair,
// 32 template points, frontier cell) and runs the same per-lane BHForce walk
// over depth-first records as the single-pair kernel. An all-pairs task is (pair, 64 template
// points, chunk of up to BATCH_CHUNK reference points): the warp stages 32
// sources at a time in shared memory and every lane adds them to its two
// points (Eq. 6).
// Epilogue launch: blocks are assigned to pairs the same way; each pair's blocks run the
// ODE step and reductions, and the pair's last block runs its rigid fit, so
// the rigid fits of all pairs run in parallel. A pair whose convergence test
// has fired skips its tasks and blocks.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>
#include <string>
#include <thread>
#include <memory>

#include "fga_batch.cuh"
#include "fga_device.cuh"
#include "fga_epi.cuh"

namespace fga {

// The k with start[k] <= x < start[k + 1], for start[0] <= x < start[n].
__device__ __forceinline__ int owner_of(const unsigned* __restrict__ start, int n, unsigned x) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (start[mid] <= x)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

#ifndef FGA_BATCH_MINBLOCKS
#define FGA_BATCH_MINBLOCKS 9  // resident blocks per SM the register budget is sized for (36 warps)
#endif
__global__ void __launch_bounds__(BATCH_WARPS * 32, FGA_BATCH_MINBLOCKS) k_batch_force(const PairDev* __restrict__ pairs,
                                                                     int npairs,
                                                                     const unsigned* __restrict__ task_start,
                                                                     unsigned ntasks, unsigned* ctr,
                                                                     const unsigned* __restrict__ order,
                                                                     unsigned* __restrict__ cost) {
  __shared__ float4 s_tile[BATCH_WARPS][64];  // 32 sources as (x, x, y, y), (z, z, m, m)
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (;;) {
    unsigned slot = 0;
    if (lane == 0) slot = atomicAdd(&ctr[0], 1u);
    slot = __shfl_sync(FULL, slot, 0);
    if (slot >= ntasks) break;
    unsigned task = order ? order[slot] : slot;
    if (task >= ntasks) task = slot;  // never index past the task range
    const int k = owner_of(task_start, npairs, task);
    const PairDev& P = pairs[k];
    DevState* ds = P.ds;
    if (ds->done) continue;
    const int64_t M = P.M;
    const float eps2 = P.eps2, theta2 = P.theta2;
    const unsigned local = task - task_start[k];
    const unsigned grp = local / (unsigned)P.K;
    const unsigned f = local - grp * (unsigned)P.K;
    const Xf xf = load_xf(ds);
    if (P.method == FGA_BH) {
      // 32 template points, one per lane, against frontier cell f
      const int64_t i = (int64_t)grp * BATCH_BH_GROUP + lane;
      const bool valid = i < M;
      const float3 y = place(xf, P.Y0[valid ? i : 0]);
      float hx = 0.f, hy = 0.f, hz = 0.f, lx = 0.f, ly = 0.f, lz = 0.f;
      unsigned count = 0, steps = 0;
      bh_task_pre(P.pcm, P.pls, P.front, f, y, valid, eps2, theta2, hx, hy, hz, lx, ly, lz, count, steps);
      if (cost && lane == 0) cost[task] = steps + 1u;
      if (valid) {
        P.hi[(int64_t)f * M + i] = make_float4(hx, hy, hz, 0.f);
        P.lo[(int64_t)f * M + i] = make_float4(lx, ly, lz, 0.f);
      }
      unsigned long long c = valid ? count : 0u;
      for (int off = 16; off > 0; off >>= 1) c += __shfl_down_sync(FULL, c, off);
      if (lane == 0 && c) atomicAdd(&ds->interactions, c);
    } else {
      // 64 template points, two per lane (the packed FP32 instructions serve
      // both), against reference chunk f, staged 32 sources at a time
      const int64_t i0 = (int64_t)grp * 64 + lane, i1 = i0 + 32;
      const bool v0 = i0 < M, v1 = i1 < M;
      const float3 y0 = place(xf, P.Y0[v0 ? i0 : 0]);
      const float3 y1 = place(xf, P.Y0[v1 ? i1 : 0]);
      float h0x = 0.f, h0y = 0.f, h0z = 0.f, l0x = 0.f, l0y = 0.f, l0z = 0.f;
      float h1x = 0.f, h1y = 0.f, h1z = 0.f, l1x = 0.f, l1y = 0.f, l1z = 0.f;
      const int64_t j0 = (int64_t)f * BATCH_CHUNK;
      const int64_t j1 = min(P.N, j0 + BATCH_CHUNK);
      // a 32-source tile for 64 points costs about as much as 16 Barnes-Hut walk steps
      if (cost && lane == 0) cost[task] = 16u * (unsigned)((j1 - j0 + 31) / 32) + 1u;
      const f2 nyx = f2_pack(-y0.x, -y1.x), nyy = f2_pack(-y0.y, -y1.y), nyz = f2_pack(-y0.z, -y1.z);
      const f2 e2 = f2_pack(eps2, eps2);
      for (int64_t b = j0; b < j1; b += 32) {
        const int64_t j = b + lane;
        const float4 src = j < j1 ? P.X4[j] : make_float4(0.f, 0.f, 0.f, 0.f);  // m = 0 pads
        s_tile[w][2 * lane] = make_float4(src.x, src.x, src.y, src.y);
        s_tile[w][2 * lane + 1] = make_float4(src.z, src.z, src.w, src.w);
        __syncwarp();
        f2 ax = f2_pack(0.f, 0.f), ay = ax, az = ax;
#pragma unroll 8
        for (int q = 0; q < 32; ++q) pair_term2(s_tile[w][2 * q], s_tile[w][2 * q + 1], nyx, nyy, nyz, e2, ax, ay, az);
        float p0x, p0y, p0z, p1x, p1y, p1z;
        f2_unpack(ax, p0x, p1x);
        f2_unpack(ay, p0y, p1y);
        f2_unpack(az, p0z, p1z);
        comp_add(h0x, l0x, p0x);
        comp_add(h0y, l0y, p0y);
        comp_add(h0z, l0z, p0z);
        comp_add(h1x, l1x, p1x);
        comp_add(h1y, l1y, p1y);
        comp_add(h1z, l1z, p1z);
        __syncwarp();
      }
      if (v0) {
        P.hi[(int64_t)f * M + i0] = make_float4(h0x, h0y, h0z, 0.f);
        P.lo[(int64_t)f * M + i0] = make_float4(l0x, l0y, l0z, 0.f);
      }
      if (v1) {
        P.hi[(int64_t)f * M + i1] = make_float4(h1x, h1y, h1z, 0.f);
        P.lo[(int64_t)f * M + i1] = make_float4(l1x, l1y, l1z, 0.f);
      }
    }
  }
  if (lane == 0) {
    // the last warp out resets the task counter for the next launch
    __threadfence();
    const unsigned out = atomicAdd(&ctr[1], 1u);
    if (out == gridDim.x * BATCH_WARPS - 1) {
      ctr[0] = 0u;
      ctr[1] = 0u;
      __threadfence();
    }
  }
}

// Block b belongs to pair k with block_start[k] <= b < block_start[k + 1].
__global__ void __launch_bounds__(EPI_BS) k_batch_epilogue(const PairDev* __restrict__ pairs, int npairs,
                                                           const unsigned* __restrict__ block_start) {
  const int k = owner_of(block_start, npairs, blockIdx.x);
  const int2 bm = make_int2(k, (int)(blockIdx.x - block_start[k]));
  const PairDev& P = pairs[k];
  DevState* ds = P.ds;
  if (ds->done) return;
  __shared__ bool s_last;
  __shared__ double s_red[NRED];
  const EpiCtx c = load_epi(ds);
  float r[NRED];
#pragma unroll
  for (int k = 0; k < NRED; ++k) r[k] = 0.f;
  for (int64_t i = (int64_t)bm.y * EPI_BS + threadIdx.x; i < P.M; i += (int64_t)P.nblk * EPI_BS)
    epi_point(i, P.Y0, P.hi, P.lo, P.K, P.M, P.V, P.ep, c, r);
  epi_block_partial(r, P.partials + (int64_t)bm.y * NRED);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(P.counter, 1u) == (unsigned)P.nblk - 1u);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  epi_last_reduce(P.partials, P.nblk, s_red);
  rigid_step_block(s_red, P.M, ds, P.ep, nullptr, P.inter_add);
  if (threadIdx.x == 0) {
    *P.counter = 0u;
    __threadfence();
  }
}

__global__ void k_done_flags(const PairDev* __restrict__ pairs, int n, int* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) out[k] = pairs[k].ds->done;
}

static std::atomic<int64_t> g_direct_max_n{32768};  // FGA_AUTO: all-pairs sum when N <= this

int resolve_method(const fga_params* p, int64_t N) {
  if (p->method != FGA_AUTO) return p->method;
  return N <= g_direct_max_n ? FGA_DIRECT : FGA_BH;
}

static int occupancy_grid(const void* kernel, int threads, int64_t want) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, 0) != cudaSuccess || b < 1) {
    cudaGetLastError();
    b = 1;
  }
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)b * sm_count()));
}

int batch_force_grid(unsigned ntasks) {
  return occupancy_grid((const void*)k_batch_force, BATCH_WARPS * 32,
                        ((int64_t)ntasks + BATCH_WARPS - 1) / BATCH_WARPS);
}


int launch_batch_iteration(const PairDev* d_pairs, int npairs, const unsigned* d_task_start,
                           unsigned ntasks, const unsigned* d_block_start, unsigned nblocks,
                           unsigned* d_ctr, int fgrid, cudaStream_t s,
                           const unsigned* order, unsigned* cost) {
  if (npairs <= 0) return FGA_OK;
  if (ntasks > 0) {
    k_batch_force<<<fgrid, BATCH_WARPS * 32, 0, s>>>(d_pairs, npairs, d_task_start, ntasks, d_ctr, order,
                                                     cost);
    FGA_LAUNCH_CHECK("batch force");
  }
  if (nblocks > 0) {
    k_batch_epilogue<<<nblocks, EPI_BS, 0, s>>>(d_pairs, npairs, d_block_start);
    FGA_LAUNCH_CHECK("batch epilogue");
  }
  return FGA_OK;
}

int launch_done_flags(const PairDev* d_pairs, int n, int* d_out, cudaStream_t s) {
  if (n <= 0) return FGA_OK;
  k_done_flags<<<(n + 127) / 128, 128, 0, s>>>(d_pairs, n, d_out);
  FGA_LAUNCH_CHECK("done flags");
  return FGA_OK;
}

int check_pair_flags(const int* f, const char* who, int64_t k) {
  if (f[0] || f[1] || f[2] || f[3] || !f[4]) {
    set_error(std::string(who) + ": pair " + std::to_string(k) +
              (f[4] ? " has a non-finite coordinate or a bad mass"
                    : " is degenerate (all centred coordinates equal)"));
    return FGA_EINVAL;
  }
  return FGA_OK;
}

int64_t pair_bytes_bound(int64_t N, int64_t M, int method, const fga_params* p) {
  const int64_t f4 = 16, pad = 4096;
  // preparation: staged inputs, normalised copies, masses (freed after setup)
  int64_t prep = 2 * (12 * (N + M)) + 4 * (N + M) + 8 * pad;
  int64_t keep = 3 * f4 * M + 8 * (int64_t)epilogue_blocks(M) * NRED + (int64_t)sizeof(DevState) + 8 * pad;
  if (method == FGA_BH) {
    // tree: bodies, index, keys, node arrays (<= 2N nodes: CoM, info, body
    // range, subtree size and position), depth-first records (<= 2N cells plus
    // <= N particle records), sort scratch
    const int64_t nodes = 2 * N + 64;
    int64_t tree = f4 * N + 4 * N + 8 * N + nodes * (f4 + 16 + 8 + 8) + 2 * f4 * (nodes + N) + 2 * 16 * N +
                   (int64_t)batch_front_target(N) * (int64_t)sizeof(FrontCell) + 32 * pad;
    keep += tree + 4 * M + 2 * f4 * (int64_t)batch_front_target(N) * M;
  } else {
    const int64_t K = (N + BATCH_CHUNK - 1) / BATCH_CHUNK;
    keep += f4 * N + 2 * f4 * K * M;
  }
  (void)p;
  return prep + keep;
}

int build_inputs(const fga_pair& q, const Prepared& pr, const fga_params* p, Scratch& sc,
                 fga_tree** tree, PairDev& P, double** mu0, cudaStream_t s) {
  int rc = 0;
  *tree = nullptr;
  std::memset(&P, 0, sizeof(P));
  P.method = resolve_method(p, q.N);
  P.N = q.N;
  P.M = q.M;
  float4* Y0 = nullptr;
  if (sc.alloc(&Y0, q.M) || sc.alloc(mu0, 3)) return FGA_ENOMEM;
  if (P.method == FGA_BH) {
    fga_tree* t = nullptr;
    if ((rc = tree_build(pr.Xn, pr.mXn, q.N, p->max_depth, &t, s, batch_front_target(q.N)))) return rc;
    *tree = t;
    int* perm = nullptr;
    if (sc.alloc(&perm, q.M)) return FGA_ENOMEM;
    if ((rc = pack_template(pr.Yn, pr.mYn, p->dt, q.M, true, Y0, perm, s))) return rc;
    P.pcm = pre_cm(t);
    P.pls = pre_ls(t);
    P.front = t->front;
    P.K = t->n_front;
  } else {
    float4* X4 = nullptr;
    if (sc.alloc(&X4, q.N)) return FGA_ENOMEM;
    if ((rc = pack_template(pr.Xn, pr.mXn, 0.f, q.N, false, X4, nullptr, s))) return rc;
    if ((rc = pack_template(pr.Yn, pr.mYn, p->dt, q.M, false, Y0, nullptr, s))) return rc;
    P.X4 = X4;
    P.K = (int)((q.N + BATCH_CHUNK - 1) / BATCH_CHUNK);
  }
  P.Y0 = Y0;
  return centroid4(Y0, q.M, *mu0, s);
}

// The pair's own constants (its parameters) in its descriptor.
static void fill_pair_params(const fga_params* p, PairDev& P) {
  P.ep = EpiParams{p->G, p->dt, p->eta, p->velocity_mode, (double)p->conv_tol, 0,
                   1.0 / (double)P.M, 1.0 / (double)p->dt, p->max_iter, p->dim};
  P.inter_add = P.method == FGA_BH ? 0ull : (unsigned long long)(P.N * P.M);
  P.eps2 = p->eps * p->eps;
  P.theta2 = p->theta * p->theta;
}

int build_state(const fga_params* p, const double* mu0, Scratch& sc, DevState* ds, PairDev& P,
                cudaStream_t s) {
  int rc = 0;
  const int64_t M = P.M;
  P.ds = ds;
  P.nblk = epilogue_blocks(M);
  if (sc.alloc(&P.hi, (size_t)P.K * M) || sc.alloc(&P.lo, (size_t)P.K * M) || sc.alloc(&P.V, M) ||
      sc.alloc(&P.partials, (size_t)P.nblk * NRED) || sc.alloc(&P.counter, 1))
    return FGA_ENOMEM;
  FGA_CUDA_TRY(cudaMemsetAsync(P.V, 0, sizeof(float4) * M, s));
  FGA_CUDA_TRY(cudaMemsetAsync(P.counter, 0, sizeof(unsigned), s));
  if ((rc = launch_state_init(ds, mu0, s))) return rc;
  // no iterations at all: the pair starts finished (max_iter = 0 in EpiParams
  // would mean "no limit")
  if (p->max_iter <= 0) FGA_CUDA_TRY(cudaMemsetAsync(&ds->done, 1, sizeof(int), s));
  fill_pair_params(p, P);
  return FGA_OK;
}

__global__ void k_states_init(DevState* __restrict__ ds, const double* const* __restrict__ mu0,
                              const int* __restrict__ done, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) state_init(ds + k, mu0[k], done[k]);
}

int build_pair(const fga_pair& q, const Prepared& pr, const fga_params* p, Scratch& sc,
               fga_tree** tree, DevState* ds, PairDev& P, cudaStream_t s) {
  double* mu0 = nullptr;
  const int rc = build_inputs(q, pr, p, sc, tree, P, &mu0, s);
  return rc ? rc : build_state(p, mu0, sc, ds, P, s);
}

void fill_pair_result(const DevState& h, const double* info, int method, const fga_params* p,
                      fga_pair_result& r) {
  std::memset(&r, 0, sizeof(r));
  std::memcpy(r.R, h.R, sizeof(r.R));
  if (p->normalize)
    fga_denormalize(h.R, h.t, info, p->a, r.t);
  else
    std::memcpy(r.t, h.t, sizeof(r.t));
  r.method = method;
  r.iterations = h.iter;
  r.converged = h.converged;
  r.interactions = (int64_t)h.interactions;
  r.status = h.status ? FGA_EINTERNAL : (h.degenerate ? FGA_EDEGENERATE : FGA_OK);
}

bool batch_layout(const std::vector<PairDev>& pairs, std::vector<unsigned>& task_start,
                  std::vector<unsigned>& block_start) {
  task_start.assign(pairs.size() + 1, 0u);
  block_start.assign(pairs.size() + 1, 0u);
  int64_t nt = 0, nb = 0;
  for (size_t k = 0; k < pairs.size(); ++k) {
    const int64_t gs = pairs[k].method == FGA_BH ? BATCH_BH_GROUP : 64;  // template points per task
    nt += (pairs[k].M + gs - 1) / gs * (int64_t)pairs[k].K;
    nb += pairs[k].nblk;
    if (nt >= ((int64_t)1 << 31) || nb >= ((int64_t)1 << 31)) return false;
    task_start[k + 1] = (unsigned)nt;
    block_start[k + 1] = (unsigned)nb;
  }
  return true;
}

}  // namespace fga

using namespace fga;

extern "C" int64_t fga_direct_max_n(int64_t new_value) {
  return new_value > 0 ? g_direct_max_n.exchange(new_value) : g_direct_max_n.load();
}

namespace {

// One host worker of the batch preparation: its stream, arena and trees.
struct PrepWorker {
  cudaStream_t st = nullptr;
  std::unique_ptr<Scratch> sc;
  std::vector<fga_tree*> trees;
  int64_t h2d = 0;
  int rc = 0;
  std::string msg;
  int start(cudaEvent_t ready) {
    FGA_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    FGA_CUDA_TRY(cudaStreamWaitEvent(st, ready, 0));
    sc.reset(new Scratch(st));
    return FGA_OK;
  }
  ~PrepWorker() {
    for (fga_tree* t : trees) fga_tree_destroy(t);
    sc.reset();
    if (st) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
  }
};

}  // namespace

extern "C" int fga_register_batch(const fga_pair* pairs, int count, const fga_params* p,
                                  fga_pair_result* results, fga_stats* stats, void* stream) {
  clear_error();
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = (cudaStream_t)stream;
  if (!pairs || count <= 0 || !results) {
    set_error("fga_register_batch: bad arguments");
    return FGA_EINVAL;
  }
  int rc = check_register_params(p);
  if (rc) return rc;
  // each pair's parameters: its own, or the call's
  std::vector<const fga_params*> pp(count);
  int iters = 0;
  for (int k = 0; k < count; ++k) {
    const fga_pair& q = pairs[k];
    if (!q.X || !q.Y || q.N <= 0 || q.M <= 0 || q.N > ((int64_t)1 << 26) || q.M > ((int64_t)1 << 26)) {
      set_error("fga_register_batch: bad sizes or null points in pair " + std::to_string(k));
      return FGA_EINVAL;
    }
    pp[k] = q.params ? q.params : p;
    if (q.params && (rc = check_register_params(q.params))) {
      set_error("fga_register_batch: parameters of pair " + std::to_string(k) + ": " + fga_last_error());
      return rc;
    }
    iters = std::max(iters, pp[k]->max_iter);
  }
  Scratch sc(s);
  // Pairs with the same inputs and the same input-shaping parameters (e.g.
  // the cells of a parameter grid over one pair) share one preparation: the
  // normalised clouds, masses, tree or packed reference and packed template.
  std::vector<int> src(count);
  {
    std::map<std::vector<uint64_t>, int> first;
    for (int k = 0; k < count; ++k) {
      const fga_pair& q = pairs[k];
      const fga_params* pk = pp[k];
      const int method = resolve_method(pk, q.N);
      auto bits = [](float f) {
        uint32_t u;
        std::memcpy(&u, &f, 4);
        return (uint64_t)u;
      };
      const std::vector<uint64_t> key = {
          (uint64_t)(uintptr_t)q.X, (uint64_t)q.N, (uint64_t)(uintptr_t)q.Y, (uint64_t)q.M,
          (uint64_t)(uintptr_t)q.mX, (uint64_t)(uintptr_t)q.mY, (uint64_t)pk->normalize,
          pk->normalize ? bits(pk->a) : 0, pk->normalize ? bits(pk->b) : 0, (uint64_t)pk->mass_mode,
          pk->mass_mode == FGA_MASS_NIV ? (uint64_t)pk->lattice : 0, bits(pk->dt), (uint64_t)method,
          method == FGA_BH ? (uint64_t)pk->max_depth : 0, (uint64_t)pk->dim};
      src[k] = first.emplace(key, k).first->second;
    }
  }
  int64_t h2d = 0;
  std::vector<Prepared> prep(count);
  std::vector<PairDev> host(count);
  std::vector<double*> mu0(count, nullptr);
  DevState* dsarr = nullptr;
  if (sc.alloc(&dsarr, (size_t)count)) return FGA_ENOMEM;
  // Preparation of the distinct inputs (normalisation, masses, checks, tree
  // or packed reference, packed template) in parallel: host workers with a
  // stream and an arena each, so that one pair's tree build (which waits for
  // the GPU between its levels) does not hold up the others. Every output
  // slot is written by exactly one worker; each worker's memory lives until
  // the call returns, after the iteration graph has finished.
  std::vector<int> uniq;
  for (int k = 0; k < count; ++k)
    if (src[k] == k) uniq.push_back(k);
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const int nw = (int)std::min<size_t>(uniq.size(), std::min(8u, hw));
  std::vector<std::unique_ptr<PrepWorker>> workers;
  {
    int dev = 0;
    FGA_CUDA_TRY(cudaGetDevice(&dev));
    cudaEvent_t ready = nullptr;
    FGA_CUDA_TRY(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    struct EvFree {
      cudaEvent_t e;
      ~EvFree() { cudaEventDestroy(e); }
    } evfree{ready};
    FGA_CUDA_TRY(cudaEventRecord(ready, s));  // inputs the caller wrote on s
    for (int w = 0; w < nw; ++w) workers.emplace_back(new PrepWorker);
    auto work = [&](int w) {
      PrepWorker& W = *workers[w];
      cudaSetDevice(dev);
      clear_error();
      W.rc = W.start(ready);
      std::vector<int> mine;
      for (size_t u = w; u < uniq.size() && !W.rc; u += nw) mine.push_back(uniq[u]);
      for (int k : mine) {
        if (W.rc) break;
        const fga_pair& q = pairs[k];
        W.rc = prepare_inputs(*W.sc, q.X, q.N, q.Y, q.M, q.mX, q.mY, pp[k], prep[k], W.h2d, W.st);
      }
      std::vector<int> flags((size_t)8 * mine.size());
      for (size_t j = 0; j < mine.size() && !W.rc; ++j)
        if (cudaMemcpyAsync(&flags[8 * j], prep[mine[j]].flags, 8 * sizeof(int), cudaMemcpyDeviceToHost,
                            W.st) != cudaSuccess) {
          set_error("fga_register_batch: reading the input checks failed");
          W.rc = FGA_ECUDA;
        }
      if (!W.rc && cudaStreamSynchronize(W.st) != cudaSuccess) {
        set_error("fga_register_batch: input preparation failed on the device");
        W.rc = FGA_ECUDA;
      }
      for (size_t j = 0; j < mine.size() && !W.rc; ++j)
        W.rc = check_pair_flags(&flags[8 * j], "fga_register_batch", mine[j]);
      for (int k : mine) {
        if (W.rc) break;
        fga_tree* t = nullptr;
        W.rc = build_inputs(pairs[k], prep[k], pp[k], *W.sc, &t, host[k], &mu0[k], W.st);
        if (t) W.trees.push_back(t);
      }
      if (!W.rc && cudaStreamSynchronize(W.st) != cudaSuccess) {
        set_error("fga_register_batch: input preparation failed on the device");
        W.rc = FGA_ECUDA;
      }
      if (W.rc) W.msg = fga_last_error();
    };
    std::vector<std::thread> threads;
    for (int w = 1; w < nw; ++w) threads.emplace_back(work, w);
    if (nw > 0) work(0);
    for (auto& t : threads) t.join();
  }
  for (auto& W : workers) {
    h2d += W->h2d;
    if (W->rc && !rc) {
      rc = W->rc;
      set_error(W->msg);
    }
  }
  if (rc) return rc;
  // every pair's own state, velocities, partial sums and block counter in
  // five allocations and one initialisation launch
  {
    size_t nhl = 0, nv = 0, npart = 0;
    for (int k = 0; k < count; ++k) {
      host[k] = host[src[k]];
      host[k].nblk = epilogue_blocks(host[k].M);
      nhl += (size_t)host[k].K * host[k].M;
      nv += (size_t)host[k].M;
      npart += (size_t)host[k].nblk * NRED;
    }
    float4 *hi = nullptr, *lo = nullptr, *V = nullptr;
    double* part = nullptr;
    unsigned* ctr = nullptr;
    if (sc.alloc(&hi, nhl) || sc.alloc(&lo, nhl) || sc.alloc(&V, nv) || sc.alloc(&part, npart) ||
        sc.alloc(&ctr, (size_t)count))
      return FGA_ENOMEM;
    FGA_CUDA_TRY(cudaMemsetAsync(V, 0, sizeof(float4) * nv, s));
    FGA_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(unsigned) * count, s));
    std::vector<const double*> mu0k(count);
    std::vector<int> donek(count);
    size_t ohl = 0, ov = 0, op = 0;
    for (int k = 0; k < count; ++k) {
      PairDev& P = host[k];
      P.ds = dsarr + k;
      P.hi = hi + ohl;
      P.lo = lo + ohl;
      P.V = V + ov;
      P.partials = part + op;
      P.counter = ctr + k;
      ohl += (size_t)P.K * P.M;
      ov += (size_t)P.M;
      op += (size_t)P.nblk * NRED;
      fill_pair_params(pp[k], P);
      mu0k[k] = mu0[src[k]];
      // no iterations at all: the pair starts finished (max_iter = 0 in
      // EpiParams would mean "no limit")
      donek[k] = pp[k]->max_iter <= 0 ? 1 : 0;
    }
    const double** d_mu0 = nullptr;
    int* d_done = nullptr;
    if (sc.alloc(&d_mu0, (size_t)count) || sc.alloc(&d_done, (size_t)count)) return FGA_ENOMEM;
    FGA_CUDA_TRY(cudaMemcpyAsync(d_mu0, mu0k.data(), sizeof(double*) * count, cudaMemcpyHostToDevice, s));
    FGA_CUDA_TRY(cudaMemcpyAsync(d_done, donek.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s));
    k_states_init<<<(count + 127) / 128, 128, 0, s>>>(dsarr, d_mu0, d_done, count);
    FGA_LAUNCH_CHECK("states_init");
    count_launch(1);
  }
  // Barnes-Hut pairs (usually the heaviest tasks) are handed out first
  std::vector<PairDev> order;
  for (int pass = 0; pass < 2; ++pass)
    for (int k = 0; k < count; ++k)
      if ((host[k].method == FGA_BH) == (pass == 0)) order.push_back(host[k]);
  std::vector<unsigned> task_start, block_start;
  if (!batch_layout(order, task_start, block_start)) {
    set_error("fga_register_batch: too many tasks in one batch (2^31)");
    return FGA_EINVAL;
  }
  PairDev* d_pairs = nullptr;
  unsigned *d_tstart = nullptr, *d_bstart = nullptr, *d_ctr = nullptr, *d_cost = nullptr, *d_order = nullptr;
  if (sc.alloc(&d_pairs, (size_t)count) || sc.alloc(&d_tstart, (size_t)count + 1) ||
      sc.alloc(&d_bstart, (size_t)count + 1) || sc.alloc(&d_ctr, 2) ||
      sc.alloc(&d_cost, (size_t)task_start[count] + 1) ||
      sc.alloc(&d_order, (size_t)task_start[count] + 1 + TASK_ORDER_SCRATCH))
    return FGA_ENOMEM;
  FGA_CUDA_TRY(cudaMemcpyAsync(d_pairs, order.data(), sizeof(PairDev) * count, cudaMemcpyHostToDevice, s));
  FGA_CUDA_TRY(cudaMemcpyAsync(d_tstart, task_start.data(), sizeof(unsigned) * (count + 1),
                               cudaMemcpyHostToDevice, s));
  FGA_CUDA_TRY(cudaMemcpyAsync(d_bstart, block_start.data(), sizeof(unsigned) * (count + 1),
                               cudaMemcpyHostToDevice, s));
  FGA_CUDA_TRY(cudaMemsetAsync(d_ctr, 0, 2 * sizeof(unsigned), s));
  const auto t_setup = std::chrono::steady_clock::now();
  // the iteration loop as one CUDA graph on a private stream ordered after s
  const unsigned ntasks = task_start[count], nblocks = block_start[count];
  const int fgrid = batch_force_grid(ntasks);
  // iteration `it`: the force launch (heavy-first task order from the second
  // iteration on, refreshed on the bh_reorder_due schedule), then the epilogue
  bool have_order = false;  // d_order is written (by an earlier launch on the same stream)
  auto force = [&](int it, cudaStream_t st) -> int {
    int r = launch_batch_iteration(d_pairs, count, d_tstart, ntasks, d_bstart, 0, d_ctr, fgrid, st, have_order ? d_order : nullptr, d_cost);
    if (r == FGA_OK && bh_reorder_due(it + 1, FGA_BATCH_REORDER_EVERY)) {
      r = launch_task_order(d_cost, ntasks, d_order, st);
      have_order = true;
      count_launch(1);
    }
    return r;
  };
  auto epilogue = [&](cudaStream_t st) -> int {
    return launch_batch_iteration(d_pairs, count, d_tstart, 0, d_bstart, nblocks, d_ctr, fgrid, st);
  };
  cudaStream_t cs = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  struct GraphCleanup {
    cudaStream_t& cs;
    cudaEvent_t& a;
    cudaEvent_t& b;
    cudaGraph_t& g;
    cudaGraphExec_t& e;
    ~GraphCleanup() {
      // the graph may still run on an error path: finish it before the
      // memory it uses is released
      if (cs) cudaStreamSynchronize(cs);
      if (e) cudaGraphExecDestroy(e);
      if (g) cudaGraphDestroy(g);
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
      if (cs) cudaStreamDestroy(cs);
    }
  } gclean{cs, ev_in, ev_out, graph, exec};
  FGA_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  FGA_CUDA_TRY(cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming));
  FGA_CUDA_TRY(cudaEventCreateWithFlags(&ev_out, cudaEventDisableTiming));
  FGA_CUDA_TRY(cudaEventRecord(ev_in, s));
  FGA_CUDA_TRY(cudaStreamWaitEvent(cs, ev_in, 0));
  double prof_ms = 0.0;
  int prof_launches = 0;
  if (iters > 0 && p->profile) {
    // profiling: plain launches with a pair of events around every force launch
    std::vector<cudaEvent_t> evs((size_t)2 * iters, nullptr);
    struct EvCleanup {
      std::vector<cudaEvent_t>& v;
      ~EvCleanup() {
        for (cudaEvent_t e : v)
          if (e) cudaEventDestroy(e);
      }
    } evclean{evs};
    for (auto& e : evs) FGA_CUDA_TRY(cudaEventCreate(&e));
    for (int it = 0; it < iters; ++it) {
      FGA_CUDA_TRY(cudaEventRecord(evs[2 * it], cs));
      if ((rc = force(it, cs))) return rc;
      FGA_CUDA_TRY(cudaEventRecord(evs[2 * it + 1], cs));
      if ((rc = epilogue(cs))) return rc;
      count_launch(2);
    }
    FGA_CUDA_TRY(cudaStreamSynchronize(cs));
    for (int it = 0; it < iters; ++it) {
      float ms = 0.f;
      FGA_CUDA_TRY(cudaEventElapsedTime(&ms, evs[2 * it], evs[2 * it + 1]));
      prof_ms += ms;
    }
    prof_launches = iters;
  } else if (iters > 0) {
    FGA_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    int lrc = FGA_OK;
    for (int it = 0; it < iters && lrc == FGA_OK; ++it) {
      lrc = force(it, cs);
      if (lrc == FGA_OK) lrc = epilogue(cs);
      count_launch(2);
    }
    cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    if (lrc != FGA_OK || ce != cudaSuccess) {
      set_error(std::string("fga_register_batch: graph capture failed: ") +
                cudaGetErrorString(ce != cudaSuccess ? ce : cudaGetLastError()));
      return FGA_ECUDA;
    }
    FGA_CUDA_TRY(cudaGraphInstantiate(&exec, graph, 0));
    FGA_CUDA_TRY(cudaGraphLaunch(exec, cs));
  }
  FGA_CUDA_TRY(cudaEventRecord(ev_out, cs));
  FGA_CUDA_TRY(cudaStreamWaitEvent(s, ev_out, 0));
  std::vector<DevState> hs(count);
  std::vector<double> infos((size_t)8 * count);
  FGA_CUDA_TRY(cudaMemcpyAsync(hs.data(), dsarr, sizeof(DevState) * count, cudaMemcpyDeviceToHost, s));
  for (int k = 0; k < count; ++k)
    if (src[k] == k)
      FGA_CUDA_TRY(cudaMemcpyAsync(&infos[8 * k], prep[k].info, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
  FGA_CUDA_TRY(cudaStreamSynchronize(s));
  const auto t_end = std::chrono::steady_clock::now();
  int code = FGA_OK;
  int64_t total = 0;
  for (int k = 0; k < count; ++k) {
    fill_pair_result(hs[k], &infos[8 * src[k]], host[k].method, pp[k], results[k]);
    if (results[k].status == FGA_EINTERNAL) code = FGA_EINTERNAL;
    else if (results[k].status == FGA_EDEGENERATE && code == FGA_OK) code = FGA_EDEGENERATE;
    total += results[k].interactions;
  }
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->iterations = iters;
    stats->interactions = total;
    stats->status = code;
    stats->h2d_bytes = h2d;
    stats->d2h_bytes = (int64_t)(sizeof(DevState) + 8 * sizeof(double) + 8 * sizeof(int)) * count;
    stats->elapsed_ms = std::chrono::duration<double, std::milli>(t_end - t0).count();
    // force time: summed event times of the force launches when profiling,
    // else the host time of the whole iteration loop
    stats->force_ms = p->profile ? prof_ms : std::chrono::duration<double, std::milli>(t_end - t_setup).count();
    stats->force_launches = prof_launches;
  }
  if (code == FGA_EINTERNAL) set_error("fga_register_batch: a device check failed in some pair");
  return code;
}
