// Autotuner: measures, on this GPU, the launch shapes and the method choice
// that the executors otherwise take from built-in defaults.
//
//   * Tile shape of the all-pairs kernel (threads per block x template points
//     per thread) for each template-size class, timed on synthetic clouds of
//     that class; the fastest shape goes into the tile table of plan_direct.
//   * The FGA_AUTO crossover between the all-pairs sum and Barnes-Hut in the
//     batch kernels: for reference sizes N = 1k .. 64k, the force cost per
//     template point of each method (a template of at least 32k points, large
//     enough that one pair fills the GPU with either method) plus, for
//     Barnes-Hut, the tree build amortised over the iterations of a
//     registration with M = N. The crossover is the largest
//     N up to which the all-pairs sum is not slower.
//
// The synthetic clouds are points on a few planar patches with a little
// noise, drawn on the device from a counter-based hash (SplitMix64's output
// mixer applied to seed and index), in the normalised box [-4, 4]^3.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include "fga_batch.cuh"

namespace fga {
namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ float unit(uint64_t h) { return (float)(h >> 40) * (1.0f / 16777216.0f); }

// n points on 8 patches (axis-aligned planes of random extent and offset).
__global__ void k_gen_cloud(float* __restrict__ out, int64_t n, uint64_t seed) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t h0 = mix64(seed * 0x9e3779b97f4a7c15ull + (uint64_t)i);
    const int patch = (int)(h0 & 7u);
    const uint64_t hp = mix64(seed + 0x1234567ull * (uint64_t)(patch + 1));
    const int axis = patch % 3;
    const float off = -3.f + 6.f * unit(hp);
    const float cu = -2.f + 4.f * unit(mix64(hp + 1)), cv = -2.f + 4.f * unit(mix64(hp + 2));
    const float su = 0.5f + 1.5f * unit(mix64(hp + 3)), sv = 0.5f + 1.5f * unit(mix64(hp + 4));
    const float u = cu + su * (unit(mix64(h0 + 11)) - 0.5f);
    const float v = cv + sv * (unit(mix64(h0 + 12)) - 0.5f);
    const float w = off + 0.02f * (unit(mix64(h0 + 13)) - 0.5f);
    float p[3];
    p[axis] = w;
    p[(axis + 1) % 3] = u;
    p[(axis + 2) % 3] = v;
    out[3 * i] = p[0];
    out[3 * i + 1] = p[1];
    out[3 * i + 2] = p[2];
  }
}

__global__ void k_fill(float* __restrict__ out, int64_t n, float v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = v;
}

int gen_cloud(float* out, int64_t n, uint64_t seed, cudaStream_t s) {
  k_gen_cloud<<<grid_for(n), 256, 0, s>>>(out, n, seed);
  FGA_LAUNCH_CHECK("gen_cloud");
  return FGA_OK;
}

int fill(float* out, int64_t n, float v, cudaStream_t s) {
  k_fill<<<grid_for(n), 256, 0, s>>>(out, n, v);
  FGA_LAUNCH_CHECK("fill");
  return FGA_OK;
}

// Times `body` (which queues work on s): one warm-up run, then the fastest of
// `reps` runs, in ms.
template <class F>
int time_min(cudaStream_t s, int reps, F body, double* ms_out) {
  cudaEvent_t a = nullptr, b = nullptr;
  struct Ev {
    cudaEvent_t& a;
    cudaEvent_t& b;
    ~Ev() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } ev{a, b};
  FGA_CUDA_TRY(cudaEventCreate(&a));
  FGA_CUDA_TRY(cudaEventCreate(&b));
  int rc = body();
  if (rc) return rc;
  double best = 1e30;
  for (int r = 0; r < reps; ++r) {
    FGA_CUDA_TRY(cudaEventRecord(a, s));
    if ((rc = body())) return rc;
    FGA_CUDA_TRY(cudaEventRecord(b, s));
    FGA_CUDA_TRY(cudaEventSynchronize(b));
    float ms = 0.f;
    FGA_CUDA_TRY(cudaEventElapsedTime(&ms, a, b));
    best = std::min(best, (double)ms);
  }
  *ms_out = best;
  return FGA_OK;
}

// A synthetic prepared pair: clouds in the normalised box, uniform masses.
int synthetic_pair(Scratch& sc, int64_t N, int64_t M, uint64_t seed, float dt, Prepared& pr, cudaStream_t s) {
  int rc = 0;
  if (sc.alloc(&pr.Xn, 3 * N) || sc.alloc(&pr.Yn, 3 * M) || sc.alloc(&pr.mXn, N) || sc.alloc(&pr.mYn, M))
    return FGA_ENOMEM;
  if ((rc = gen_cloud(pr.Xn, N, seed, s)) || (rc = gen_cloud(pr.Yn, M, seed + 1, s)) ||
      (rc = fill(pr.mXn, N, (float)(1.0 / (double)N), s)) || (rc = fill(pr.mYn, M, dt, s)))
    return rc;
  return FGA_OK;
}

}  // namespace
}  // namespace fga

using namespace fga;

extern "C" int fga_set_direct_tile(int size_class, int bs, int qpt) {
  clear_error();
  if (size_class < 0 || size_class > 2 || !direct_tile_supported(bs, qpt)) {
    set_error("fga_set_direct_tile: size class must be 0..2, bs 128 or 256, qpt 1, 2 or 4");
    return FGA_EINVAL;
  }
  set_direct_tile(size_class, bs, qpt);
  return FGA_OK;
}

extern "C" int fga_get_direct_tile(int size_class, int* bs, int* qpt) {
  clear_error();
  if (size_class < 0 || size_class > 2 || !bs || !qpt) {
    set_error("fga_get_direct_tile: bad arguments");
    return FGA_EINVAL;
  }
  get_direct_tile(size_class, bs, qpt);
  return FGA_OK;
}

extern "C" int fga_autotune(const fga_params* p_in, int flags, void* stream, fga_tune_report* out) {
  clear_error();
  const auto t0 = std::chrono::steady_clock::now();
  if (!out) {
    set_error("fga_autotune: null report");
    return FGA_EINVAL;
  }
  fga_params p;
  if (p_in) {
    p = *p_in;
  } else {
    fga_params_default(&p);
  }
  int rc = check_register_params(&p);
  if (rc) return rc;
  std::memset(out, 0, sizeof(*out));
  cudaStream_t s = (cudaStream_t)stream;
  const int reps = 3;

  // ---------------------------------------------------------------- direct tiles
  if (flags & FGA_TUNE_DIRECT_TILES) {
    static const int64_t classN[3] = {4096, 16384, 65536};
    static const int64_t classM[3] = {4096, 32768, 131072};
    static const int shapes[6][2] = {{128, 1}, {128, 2}, {128, 4}, {256, 1}, {256, 2}, {256, 4}};
    for (int c = 0; c < 3; ++c) {
      const int64_t N = classN[c], M = classM[c];
      Scratch sc(s);
      Prepared pr;
      float4 *X4 = nullptr, *Y0 = nullptr;
      DevState* ds = nullptr;
      double* mu0 = nullptr;
      if ((rc = synthetic_pair(sc, N, M, 77 + c, p.dt, pr, s))) return rc;
      if (sc.alloc(&X4, N) || sc.alloc(&Y0, M) || sc.alloc(&ds, 1) || sc.alloc(&mu0, 3)) return FGA_ENOMEM;
      if ((rc = pack_template(pr.Xn, pr.mXn, 0.f, N, false, X4, nullptr, s)) ||
          (rc = pack_template(pr.Yn, pr.mYn, p.dt, M, false, Y0, nullptr, s)) ||
          (rc = centroid4(Y0, M, mu0, s)) || (rc = launch_state_init(ds, mu0, s)))
        return rc;
      int old_bs = 0, old_q = 0;
      get_direct_tile(c, &old_bs, &old_q);
      double best = 1e30;
      int best_k = -1;
      for (int k = 0; k < 6; ++k) {
        set_direct_tile(c, shapes[k][0], shapes[k][1]);
        const DirectPlan plan = plan_direct(N, M);
        ForceBuffers fb;
        if (sc.alloc(&fb.hi, (size_t)plan.S * M) || sc.alloc(&fb.lo, (size_t)plan.S * M)) return FGA_ENOMEM;
        double ms = 0;
        rc = time_min(s, reps, [&] { return launch_direct(X4, N, Y0, M, ds, p.eps, plan, fb, s); }, &ms);
        if (rc) {
          set_direct_tile(c, old_bs, old_q);
          return rc;
        }
        count_launch(reps + 1);
        if (ms < best) {
          best = ms;
          best_k = k;
        }
      }
      set_direct_tile(c, shapes[best_k][0], shapes[best_k][1]);
      out->direct_bs[c] = shapes[best_k][0];
      out->direct_qpt[c] = shapes[best_k][1];
      out->direct_gips[c] = (double)N * (double)M / (best * 1e-3) / 1e9;
    }
  } else {
    for (int c = 0; c < 3; ++c) get_direct_tile(c, &out->direct_bs[c], &out->direct_qpt[c]);
  }

  // ---------------------------------------------------------------- crossover
  if (flags & FGA_TUNE_CROSSOVER) {
    const int iters = p.max_iter > 0 ? p.max_iter : 100;
    int64_t crossover = 0;
    bool bh_won = false;
    const int64_t warps = (int64_t)sm_count() * 32;
    for (int k = 0; k < FGA_TUNE_NSIZES; ++k) {
      const int64_t N = (int64_t)1024 << k;
      out->sizes[k] = N;
      // template size: at least 32768 points and enough 64-point all-pairs
      // tasks (one per reference chunk) for 4 per resident warp, so that both
      // methods fill the GPU as in a large batch
      const int64_t chunks = (N + BATCH_CHUNK - 1) / BATCH_CHUNK;
      const int64_t Mt = std::max<int64_t>(32768, (4 * warps + chunks - 1) / chunks * 64);
      double per_point[2] = {0, 0};
      for (int m = 0; m < 2; ++m) {
        fga_params q = p;
        q.method = m == 0 ? FGA_DIRECT : FGA_BH;
        Scratch sc(s);
        Prepared pr;
        if ((rc = synthetic_pair(sc, N, Mt, 1000 + k, p.dt, pr, s))) return rc;
        DevState* ds = nullptr;
        if (sc.alloc(&ds, 1)) return FGA_ENOMEM;
        fga_pair qp;
        std::memset(&qp, 0, sizeof(qp));
        qp.X = pr.Xn;
        qp.N = N;
        qp.Y = pr.Yn;
        qp.M = Mt;
        PairDev P;
        fga_tree* tree = nullptr;
        const auto tb0 = std::chrono::steady_clock::now();
        rc = build_pair(qp, pr, &q, sc, &tree, ds, P, s);
        if (rc == FGA_OK) {
          const cudaError_t e = cudaStreamSynchronize(s);
          if (e != cudaSuccess) {
            set_error(std::string("fga_autotune: ") + cudaGetErrorString(e));
            rc = FGA_ECUDA;
          }
        }
        const double build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tb0).count();
        struct TreeFree {
          fga_tree* t;
          ~TreeFree() { fga_tree_destroy(t); }
        } tf{tree};
        if (rc) return rc;
        std::vector<PairDev> one(1, P);
        std::vector<unsigned> ts, bs;
        batch_layout(one, ts, bs);
        PairDev* d_pairs = nullptr;
        unsigned *d_ts = nullptr, *d_bs = nullptr, *d_ctr = nullptr;
        if (sc.alloc(&d_pairs, 1) || sc.alloc(&d_ts, 2) || sc.alloc(&d_bs, 2) || sc.alloc(&d_ctr, 2))
          return FGA_ENOMEM;
        FGA_CUDA_TRY(cudaMemcpyAsync(d_pairs, one.data(), sizeof(PairDev), cudaMemcpyHostToDevice, s));
        FGA_CUDA_TRY(cudaMemcpyAsync(d_ts, ts.data(), 2 * sizeof(unsigned), cudaMemcpyHostToDevice, s));
        FGA_CUDA_TRY(cudaMemcpyAsync(d_bs, bs.data(), 2 * sizeof(unsigned), cudaMemcpyHostToDevice, s));
        FGA_CUDA_TRY(cudaMemsetAsync(d_ctr, 0, 2 * sizeof(unsigned), s));
        const int fgrid = batch_force_grid(ts[1]);
        double ms = 0;
        rc = time_min(s, reps, [&] {
          return launch_batch_iteration(d_pairs, 1, d_ts, ts[1], d_bs, 0, d_ctr, fgrid, s);
        }, &ms);
        if (rc) return rc;
        count_launch(reps + 1);
        // cost per template point and iteration; the tree build is spread
        // over the iterations of a registration with M = N template points
        per_point[m] = ms / (double)Mt + (m == 1 ? build_ms / ((double)iters * (double)N) : 0.0);
        if (m == 1) out->bh_build_ms[k] = build_ms;
      }
      out->direct_us_per_point[k] = 1e3 * per_point[0];
      out->bh_us_per_point[k] = 1e3 * per_point[1];
      if (!bh_won && per_point[0] <= per_point[1])
        crossover = N;
      else
        bh_won = true;
    }
    if (crossover == 0) crossover = 512;
    out->direct_max_n = crossover;
    fga_direct_max_n(crossover);
  } else {
    out->direct_max_n = fga_direct_max_n(0);
  }
  FGA_CUDA_TRY(cudaStreamSynchronize(s));
  out->elapsed_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return FGA_OK;
}
