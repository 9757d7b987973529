// C-ABI entry points of libfga (declared in include/fga.h): parameter checks,
// buffer management and the orchestration of the kernels of fga_prep.cu,
// fga_tree.cu and fga_force.cu.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "fga_internal.cuh"

// ------------------------------------------------------------------ errors, counters, pools
namespace fga {

static thread_local std::string g_err;
static std::atomic<int64_t> g_launches{0};

void set_error(const std::string& msg) { g_err = msg; }
void clear_error() { g_err.clear(); }
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

static std::mutex g_mu;
static std::map<int, cudaMemPool_t> g_pools;
static std::map<int, int> g_sms;

static cudaMemPool_t pool_for(int dev) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_pools.find(dev);
  if (it != g_pools.end()) return it->second;
  cudaMemPoolProps props;
  std::memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.handleTypes = cudaMemHandleTypeNone;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  cudaMemPool_t pool = nullptr;
  if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  uint64_t keep = UINT64_MAX;  // keep freed blocks cached for the next call
  cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  // a block freed on one stream is reused by another only once the free has
  // completed, never by making the other stream wait (the serving engine
  // prepares pairs on one stream while another runs)
  int no = 0;
  cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no);
  g_pools[dev] = pool;
  return pool;
}

int dev_alloc(void** p, size_t bytes, cudaStream_t s) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaMemPool_t pool = pool_for(dev);
  if (!pool) {
    set_error("cudaMemPoolCreate failed");
    return FGA_ECUDA;
  }
  cudaError_t e = cudaMallocFromPoolAsync(p, std::max<size_t>(bytes, 16), pool, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error(std::string("device allocation of ") + std::to_string(bytes) +
              " bytes failed: " + cudaGetErrorString(e));
    *p = nullptr;
    return e == cudaErrorMemoryAllocation ? FGA_ENOMEM : FGA_ECUDA;
  }
  return FGA_OK;
}

void dev_free(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

int sm_count() {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_sms.find(dev);
  if (it != g_sms.end()) return it->second;
  int n = 0;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
  g_sms[dev] = n;
  return n;
}

// Barnes-Hut forces are summed as 64-bit fixed-point integers whose grid is
// set by the largest possible sum, mass_total / (2.598 eps^2). The smallest
// force of a point is about mass_total / diag^2 (diag: the diagonal of the
// tree's box), so the grid's rounding, at most 2^-54 mass_total / (2.598
// eps^2) per point, stays below 2 % of the force tolerance (1e-5 of the sum of
// the term magnitudes) while diag <= 1e5 eps. Smaller eps are rejected.
static int check_bh_eps(const fga_tree* t, float eps) {
  double d2 = 0.0;
  for (int k = 0; k < 3; ++k) {
    const double e = (double)t->box_hi[k] - (double)t->box_lo[k];
    d2 += e * e;
  }
  if (std::sqrt(d2) > 1e5 * (double)eps) {
    set_error("Barnes-Hut: eps must be at least 1e-5 of the reference's bounding-box diagonal");
    return FGA_EINVAL;
  }
  return FGA_OK;
}

int check_params(const fga_params* p, bool need_tree) {
  if (!p) {
    set_error("null fga_params");
    return FGA_EINVAL;
  }
  if (!(p->eps > 0.f) || !std::isfinite(p->eps)) {
    set_error("eps must be > 0");
    return FGA_EINVAL;
  }
  if (!(p->theta >= 0.f) || !std::isfinite(p->theta)) {
    set_error("theta must be >= 0");
    return FGA_EINVAL;
  }
  if (!(p->dt > 0.f) || !std::isfinite(p->dt) || !std::isfinite(p->G) || !std::isfinite(p->eta)) {
    set_error("dt must be > 0 and G, eta finite");
    return FGA_EINVAL;
  }
  if (p->method != FGA_DIRECT && p->method != FGA_BH && p->method != FGA_AUTO) {
    set_error("method must be FGA_DIRECT, FGA_BH or FGA_AUTO");
    return FGA_EINVAL;
  }
  if (p->velocity_mode != FGA_VEL_UNCONSTRAINED && p->velocity_mode != FGA_VEL_RIGID) {
    set_error("bad velocity_mode");
    return FGA_EINVAL;
  }
  if (need_tree && (p->max_depth < 1 || p->max_depth > 20)) {
    set_error("max_depth must be in 1..20");
    return FGA_EINVAL;
  }
  if (p->dim != 2 && p->dim != 3) {
    set_error("dim must be 2 or 3");
    return FGA_EINVAL;
  }
  if (p->bh_walk < FGA_WALK_AUTO || p->bh_walk > FGA_WALK_CURSOR128) {
    set_error("bh_walk must be FGA_WALK_AUTO, _LANE, _COOP, _CURSOR, _CURSOR32 or _CURSOR128");
    return FGA_EINVAL;
  }
  if (p->max_iter < 0) {
    set_error("max_iter must be >= 0");
    return FGA_EINVAL;
  }
  return FGA_OK;
}

// Read back device flags (synchronises s).
int read_flags(const int* d_flags, int n, int* h, cudaStream_t s) {
  FGA_CUDA_TRY(cudaMemcpyAsync(h, d_flags, sizeof(int) * n, cudaMemcpyDeviceToHost, s));
  FGA_CUDA_TRY(cudaStreamSynchronize(s));
  return FGA_OK;
}

__global__ void k_pack4(const float* __restrict__ xyz, const float* __restrict__ m, float m_default,
                        int64_t n, float4* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = make_float4(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], m ? m[i] : m_default);
}

__global__ void k_gather4(const float* __restrict__ xyz, const float* __restrict__ m, float m_default,
                          int64_t n, const int* __restrict__ idx, float4* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = idx[i];
    out[i] = make_float4(xyz[3 * j], xyz[3 * j + 1], xyz[3 * j + 2], m ? m[j] : m_default);
  }
}

unsigned grid_for(int64_t n) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8 * (int64_t)sm_count()));
}

// Pack template points into float4 (x, y, z, m); with `sort`, order them along
// a Morton curve of their own bounding box (10 bits per axis) and return the
// permutation (sorted position -> original index).
int pack_template(const float* Y, const float* mY, float m_default, int64_t M, bool sort,
                         float4* Y0, int* perm, cudaStream_t s) {
  if (!sort) {
    k_pack4<<<grid_for(M), 256, 0, s>>>(Y, mY, m_default, M, Y0);
    FGA_LAUNCH_CHECK("pack4");
    return FGA_OK;
  }
  Scratch sc(s);
  unsigned long long *keys = nullptr, *ktmp = nullptr;
  int* itmp = nullptr;
  float* box = nullptr;
  int rc = sc.alloc(&keys, M) | sc.alloc(&ktmp, M) | sc.alloc(&itmp, M) | sc.alloc(&box, 6);
  if (rc) return FGA_ENOMEM;
  if ((rc = bbox_xyz(Y, M, box, box + 3, s))) return rc;
  if ((rc = morton_keys(Y, M, box, box + 3, 10, keys, perm, s))) return rc;
  if ((rc = radix_sort_pairs(keys, perm, ktmp, itmp, M, 30, s))) return rc;
  k_gather4<<<grid_for(M), 256, 0, s>>>(Y, mY, m_default, M, perm, Y0);
  FGA_LAUNCH_CHECK("gather4");
  return FGA_OK;
}

// Device pointer or host pointer? Unregistered host memory reports
// cudaMemoryTypeUnregistered; pinned host memory cudaMemoryTypeHost.
bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}


// Register-level parameter checks beyond check_params.
int check_register_params(const fga_params* p) {
  int rc = check_params(p, p && p->method != FGA_DIRECT);
  if (rc) return rc;
  if (p->normalize && !(p->b > p->a)) {
    set_error("b must exceed a");
    return FGA_EINVAL;
  }
  if (p->mass_mode != FGA_MASS_UNIFORM && p->mass_mode != FGA_MASS_NIV && p->mass_mode != FGA_MASS_KNN) {
    set_error("bad mass_mode");
    return FGA_EINVAL;
  }
  if (p->mass_mode == FGA_MASS_KNN && p->lattice != 8 && p->lattice != 16 && p->lattice != 32) {
    set_error("k (lattice) for FGA_MASS_KNN must be 8, 16 or 32");
    return FGA_EINVAL;
  }
  if (p->mass_mode == FGA_MASS_NIV && (p->lattice < 1 || p->lattice > 256)) {
    set_error("lattice must be in 1..256");
    return FGA_EINVAL;
  }
  return FGA_OK;
}

// Stage one pair on the device (host inputs are copied), check it, normalise
// it (Appendix A, if p->normalize) and assign the masses: reference masses
// sum to 1 (p->mass_mode, or the given ones rescaled), template masses have
// mean dt. No synchronisation: out.flags (8 ints) hold 1 at [0..3] for a
// non-finite coordinate or a bad mass of X, Y, mX, mY and 1 at [4] when the
// normalisation was well defined.
int prepare_inputs(Scratch& sc, const float* X, int64_t N, const float* Y, int64_t M,
                   const float* mX, const float* mY, const fga_params* p, Prepared& out,
                   int64_t& h2d, cudaStream_t s) {
  int rc = 0;
  auto stage = [&](const float* src, int64_t count, const float** dst) -> int {
    if (!src) {
      *dst = nullptr;
      return FGA_OK;
    }
    if (is_device_ptr(src)) {
      *dst = src;
      return FGA_OK;
    }
    float* d = nullptr;
    if (sc.alloc(&d, count)) return FGA_ENOMEM;
    FGA_CUDA_TRY(cudaMemcpyAsync(d, src, sizeof(float) * count, cudaMemcpyHostToDevice, s));
    h2d += (int64_t)sizeof(float) * count;
    *dst = d;
    return FGA_OK;
  };
  const float *dX = nullptr, *dY = nullptr, *dmX = nullptr, *dmY = nullptr;
  const int64_t cols = p->dim == 2 ? 2 : 3;
  if ((rc = stage(X, cols * N, &dX)) || (rc = stage(Y, cols * M, &dY)) || (rc = stage(mX, N, &dmX)) ||
      (rc = stage(mY, M, &dmY)))
    return rc;
  if (cols == 2) {
    // planar clouds: the plane z = 0 of the 3-D path
    float *eX = nullptr, *eY = nullptr;
    if (sc.alloc(&eX, 3 * N) || sc.alloc(&eY, 3 * M)) return FGA_ENOMEM;
    if ((rc = embed_planar(dX, N, eX, s)) || (rc = embed_planar(dY, M, eY, s))) return rc;
    dX = eX;
    dY = eY;
  }
  if (sc.alloc(&out.Xn, 3 * N) || sc.alloc(&out.Yn, 3 * M) || sc.alloc(&out.mXn, N) ||
      sc.alloc(&out.mYn, M) || sc.alloc(&out.info, 8) || sc.alloc(&out.flags, 8))
    return FGA_ENOMEM;
  FGA_CUDA_TRY(cudaMemsetAsync(out.flags, 0, 8 * sizeof(int), s));
  if ((rc = check_finite(dX, 3 * N, out.flags, s)) || (rc = check_finite(dY, 3 * M, out.flags + 1, s)))
    return rc;
  if (dmX && (rc = check_masses(dmX, N, out.flags + 2, s))) return rc;
  if (dmY && (rc = check_masses(dmY, M, out.flags + 3, s))) return rc;
  if (p->normalize) {
    if ((rc = normalize_device(dX, N, dY, M, p->a, p->b, out.Xn, out.Yn, out.info, out.flags + 4, s)))
      return rc;
  } else {
    static const double ident[8] = {0, 0, 0, 0, 0, 0, 0, 1};
    static const int one = 1;
    FGA_CUDA_TRY(cudaMemcpyAsync(out.Xn, dX, sizeof(float) * 3 * N, cudaMemcpyDeviceToDevice, s));
    FGA_CUDA_TRY(cudaMemcpyAsync(out.Yn, dY, sizeof(float) * 3 * M, cudaMemcpyDeviceToDevice, s));
    FGA_CUDA_TRY(cudaMemcpyAsync(out.info, ident, sizeof(ident), cudaMemcpyHostToDevice, s));
    FGA_CUDA_TRY(cudaMemcpyAsync(out.flags + 4, &one, sizeof(int), cudaMemcpyHostToDevice, s));
  }
  if (dmX)
    rc = rescale_masses(dmX, N, 1.0, out.mXn, s);
  else
    rc = masses_device(out.Xn, N, p->mass_mode, p->lattice, p->a, p->b, 1.0, out.mXn, s, p->dim == 2 ? 2 : 3);
  if (rc) return rc;
  if (dmY)
    rc = rescale_masses(dmY, M, (double)p->dt * (double)M, out.mYn, s);
  else
    rc = masses_device(out.Yn, M, FGA_MASS_UNIFORM, 1, 0.f, 1.f, (double)p->dt * (double)M, out.mYn, s);
  return rc;
}

}  // namespace fga

using namespace fga;

// ------------------------------------------------------------------ state
struct fga_state {
  fga_params p;
  int64_t N = 0, M = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  const fga_tree* tree = nullptr;
  fga_tree* own_tree = nullptr;
  float4* X4 = nullptr;
  float4* Y0 = nullptr;
  int* perm = nullptr;
  float4* V = nullptr;
  ForceBuffers fb;
  DirectPlan plan;
  DevState* ds = nullptr;
  double* partials = nullptr;
  unsigned* counter = nullptr;
  double* traj = nullptr;
  int max_traj = 0;
  int queued = 0;
  unsigned* bh_cost = nullptr;   // BH: step count of every task in the last launch
  unsigned* bh_order = nullptr;  // BH: heavy-first task order derived from bh_cost
  int bh_kind = 0;               // BH: walk of the force launch (bh_walk_kind)
  unsigned bh_ntasks = 0;
  int bh_launches = 0;
  bool bh_have_order = false;
  bool small_loop = false;       // all-pairs: the loop runs as one cluster launch (fga_small.cu)
  std::vector<cudaEvent_t> events;  // with p.profile: start/stop per force launch
  int timed = 0;                    // recorded start/stop pairs
};

extern "C" {

void fga_params_default(fga_params* p) {
  if (!p) return;
  p->G = 66.7f;
  p->eps = 0.2f;
  p->eta = 0.2f;
  p->dt = 0.1f;
  p->theta = 0.6f;
  p->max_iter = 100;
  p->conv_tol = 0.f;
  p->method = FGA_BH;
  p->normalize = 1;
  p->a = -5.f;
  p->b = 5.f;
  p->velocity_mode = FGA_VEL_UNCONSTRAINED;
  p->max_depth = 20;
  p->mass_mode = FGA_MASS_UNIFORM;
  p->lattice = 16;
  p->profile = 0;
  p->dim = 3;
  p->bh_walk = FGA_WALK_AUTO;
}

const char* fga_last_error(void) { return g_err.c_str(); }
int64_t fga_launch_count(void) { return g_launches.load(); }

void fga_denormalize(const double R[9], const double t_norm[3], const double info[8], float a,
                     double t_out[3]) {
  // X^ = s (X - Xbar - l 1) + a 1 and the same for Y; R Y^ + t_norm = X^ solved for X.
  const double l = info[6], sc = info[7], aa = (double)a;
  for (int r = 0; r < 3; ++r) {
    const double* row = R + 3 * r;
    const double r_ybar = row[0] * info[3] + row[1] * info[4] + row[2] * info[5];
    const double r_one = row[0] + row[1] + row[2];
    t_out[r] = info[r] - r_ybar + l * (1.0 - r_one) + (aa * r_one + t_norm[r] - aa) / sc;
  }
}

int fga_normalize(const float* X, int64_t N, const float* Y, int64_t M, float a, float b,
                  float* Xn_out, float* Yn_out, double info_out[8], void* stream) {
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  if (N <= 0 || M <= 0 || !(b > a) || !X || !Y || !Xn_out || !Yn_out || !info_out) {
    set_error("fga_normalize: bad arguments");
    return FGA_EINVAL;
  }
  Scratch sc(s);
  int* flags = nullptr;
  double* info = nullptr;
  float *Xc = nullptr, *Yc = nullptr;
  if (sc.alloc(&flags, 2) || sc.alloc(&info, 8) || sc.alloc(&Xc, 3 * N) || sc.alloc(&Yc, 3 * M))
    return FGA_ENOMEM;
  FGA_CUDA_TRY(cudaMemsetAsync(flags, 0, 2 * sizeof(int), s));
  int rc = check_finite(X, 3 * N, flags, s);
  if (!rc) rc = check_finite(Y, 3 * M, flags, s);
  // the outputs may alias the inputs: work from copies
  if (!rc) {
    FGA_CUDA_TRY(cudaMemcpyAsync(Xc, X, sizeof(float) * 3 * N, cudaMemcpyDeviceToDevice, s));
    FGA_CUDA_TRY(cudaMemcpyAsync(Yc, Y, sizeof(float) * 3 * M, cudaMemcpyDeviceToDevice, s));
    rc = normalize_device(Xc, N, Yc, M, a, b, Xn_out, Yn_out, info, flags + 1, s);
  }
  if (rc) return rc;
  int h[2];
  FGA_CUDA_TRY(cudaMemcpyAsync(info_out, info, sizeof(double) * 8, cudaMemcpyDeviceToHost, s));
  if ((rc = read_flags(flags, 2, h, s))) return rc;
  if (h[0]) {
    set_error("fga_normalize: non-finite input coordinate");
    return FGA_EINVAL;
  }
  if (!h[1]) {
    set_error("fga_normalize: degenerate input (all centred coordinates equal)");
    return FGA_EINVAL;
  }
  return FGA_OK;
}

int fga_masses(const float* pts, int64_t n, int mode, int lattice, float a, float b, double total,
               float* masses_out, void* stream) {
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  if (n <= 0 || !pts || !masses_out || !(total > 0) || !std::isfinite(total) ||
      (mode != FGA_MASS_UNIFORM && mode != FGA_MASS_NIV && mode != FGA_MASS_KNN) ||
      (mode == FGA_MASS_NIV && (lattice < 1 || lattice > 256 || !(b > a))) ||
      (mode == FGA_MASS_KNN && ((lattice != 8 && lattice != 16 && lattice != 32) || n <= lattice || !(b > a)))) {
    set_error("fga_masses: bad arguments");
    return FGA_EINVAL;
  }
  return masses_device(pts, n, mode, lattice, a, b, total, masses_out, s);
}

int fga_tree_build(const float* X, const float* mX, int64_t N, const fga_params* p, fga_tree** out,
                   void* stream) {
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  if (!out || !X || N <= 0 || N > (int64_t)1 << 26 || !p || p->max_depth < 1 || p->max_depth > 20) {
    set_error("fga_tree_build: bad arguments (1 <= N <= 2^26, max_depth 1..20)");
    return FGA_EINVAL;
  }
  *out = nullptr;
  Scratch sc(s);
  int* flags = nullptr;
  if (sc.alloc(&flags, 2)) return FGA_ENOMEM;
  FGA_CUDA_TRY(cudaMemsetAsync(flags, 0, 2 * sizeof(int), s));
  int rc = check_finite(X, 3 * N, flags, s);
  if (!rc && mX) rc = check_masses(mX, N, flags + 1, s);
  if (rc) return rc;
  int h[2];
  if ((rc = read_flags(flags, 2, h, s))) return rc;
  if (h[0] || h[1]) {
    set_error("fga_tree_build: non-finite coordinate or negative/non-finite mass");
    return FGA_EINVAL;
  }
  return tree_build(X, mX, N, p->max_depth, out, s);
}

int fga_forces(const fga_tree* tree, const float* X, const float* mX, int64_t N, const float* Y,
               const float* mY, int64_t M, const fga_params* p, float* acc_out,
               int64_t* interactions_out, void* stream) {
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  if (!p || !(p->eps > 0.f) || !(p->theta >= 0.f) || M <= 0 || !Y || !acc_out ||
      (!tree && (N <= 0 || !X))) {
    set_error("fga_forces: bad arguments");
    return FGA_EINVAL;
  }
  if (tree && check_bh_eps(tree, p->eps)) return FGA_EINVAL;
  Scratch sc(s);
  float4 *Y0 = nullptr, *X4 = nullptr;
  int* perm = nullptr;
  DevState* ds = nullptr;
  ForceBuffers fb;
  DirectPlan plan;
  int rc = sc.alloc(&Y0, M) | sc.alloc(&ds, 1);
  if (rc) return FGA_ENOMEM;
  if (tree) {
    if (sc.alloc(&perm, M) || sc.alloc(&fb.acc, (size_t)3 * M)) return FGA_ENOMEM;
    FGA_CUDA_TRY(cudaMemsetAsync(fb.acc, 0, sizeof(long long) * 3 * M, s));
    rc = pack_template(Y, mY, 1.0f, M, true, Y0, perm, s);
  } else {
    if (sc.alloc(&X4, N)) return FGA_ENOMEM;
    rc = pack_template(Y, mY, 1.0f, M, false, Y0, nullptr, s);
    if (!rc) {
      k_pack4<<<grid_for(N), 256, 0, s>>>(X, mX, (float)(1.0 / (double)N), N, X4);
      FGA_LAUNCH_CHECK("pack4 X");
    }
    plan = plan_direct(N, M);
    fb.S = plan.S;
  }
  if (rc) return rc;
  if (!tree && (sc.alloc(&fb.hi, (size_t)fb.S * M) || sc.alloc(&fb.lo, (size_t)fb.S * M))) return FGA_ENOMEM;
  if ((rc = launch_state_init(ds, nullptr, s))) return rc;
  if (tree)
    rc = launch_bh(tree, Y0, M, ds, p->eps, p->theta, fb, s, bh_walk_kind(M, p->bh_walk));
  else
    rc = launch_direct(X4, N, Y0, M, ds, p->eps, plan, fb, s);
  if (rc) return rc;
  if ((rc = launch_forces_out(fb, M, Y0, mY != nullptr, p->G, perm, acc_out, s))) return rc;
  if (interactions_out) {
    DevState h;
    FGA_CUDA_TRY(cudaMemcpyAsync(&h, ds, sizeof(h), cudaMemcpyDeviceToHost, s));
    FGA_CUDA_TRY(cudaStreamSynchronize(s));
    *interactions_out = tree ? (int64_t)h.interactions : N * M;
  }
  return FGA_OK;
}

__global__ void k_terms_out(const unsigned* __restrict__ terms, const int* __restrict__ perm, int64_t M,
                            int32_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M;
       i += (int64_t)gridDim.x * blockDim.x)
    out[perm[i]] = (int32_t)terms[i];
}

int fga_forces_terms(const fga_tree* tree, const float* Y, const float* mY, int64_t M,
                     const fga_params* p, float* acc_out, int32_t* terms_out, void* stream) {
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  if (!tree || !p || !(p->eps > 0.f) || !(p->theta >= 0.f) || M <= 0 || !Y || !acc_out || !terms_out) {
    set_error("fga_forces_terms: bad arguments");
    return FGA_EINVAL;
  }
  if (check_bh_eps(tree, p->eps)) return FGA_EINVAL;
  Scratch sc(s);
  float4* Y0 = nullptr;
  int* perm = nullptr;
  unsigned* terms = nullptr;
  DevState* ds = nullptr;
  ForceBuffers fb;
  if (sc.alloc(&Y0, M) || sc.alloc(&ds, 1) || sc.alloc(&perm, M) || sc.alloc(&terms, M))
    return FGA_ENOMEM;
  int rc = pack_template(Y, mY, 1.0f, M, true, Y0, perm, s);
  if (rc) return rc;
  if (sc.alloc(&fb.acc, (size_t)3 * M)) return FGA_ENOMEM;
  FGA_CUDA_TRY(cudaMemsetAsync(fb.acc, 0, sizeof(long long) * 3 * M, s));
  FGA_CUDA_TRY(cudaMemsetAsync(terms, 0, sizeof(unsigned) * M, s));
  if ((rc = launch_state_init(ds, nullptr, s))) return rc;
  rc = launch_bh(tree, Y0, M, ds, p->eps, p->theta, fb, s, bh_walk_kind(M, p->bh_walk), nullptr, nullptr,
                 terms);
  if (rc) return rc;
  if ((rc = launch_forces_out(fb, M, Y0, mY != nullptr, p->G, perm, acc_out, s))) return rc;
  k_terms_out<<<grid_for(M), 256, 0, s>>>(terms, perm, M, terms_out);
  FGA_LAUNCH_CHECK("terms_out");
  return FGA_OK;
}

}  // extern "C"

// Build a state from device arrays that are already checked.
static int state_create_checked(const float* Xn, const float* mX, int64_t N, const float* Yn,
                                const float* mY, int64_t M, const fga_tree* tree,
                                const fga_params* p, fga_state** out, cudaStream_t s) {
  fga_state* st = new fga_state();
  st->p = *p;
  st->N = N;
  st->M = M;
  st->stream = s;
  cudaGetDevice(&st->device);
  auto fail = [&](int code) {
    fga_state_destroy(st);
    return code;
  };
  const bool bh = p->method == FGA_BH;
  int rc = 0;
  if (bh) {
    if (tree) {
      st->tree = tree;
    } else {
      if ((rc = tree_build(Xn, mX, N, p->max_depth, &st->own_tree, s))) return fail(rc);
      st->tree = st->own_tree;
    }
    if ((rc = check_bh_eps(st->tree, p->eps))) return fail(rc);
  } else {
    if (dev_alloc_n(&st->X4, N, s)) return fail(FGA_ENOMEM);
    k_pack4<<<grid_for(N), 256, 0, s>>>(Xn, mX, (float)(1.0 / (double)N), N, st->X4);
    FGA_LAUNCH_CHECK("pack4 X");
    st->plan = plan_direct(N, M);
    st->fb.S = st->plan.S;
    st->small_loop = small_loop_eligible(N, M, st->plan) && small_loop_available(st->plan);
  }
  if (dev_alloc_n(&st->Y0, M, s) || dev_alloc_n(&st->V, M, s) || dev_alloc_n(&st->ds, 1, s) ||
      dev_alloc_n(&st->counter, 1, s))
    return fail(FGA_ENOMEM);
  if (bh && dev_alloc_n(&st->perm, M, s)) return fail(FGA_ENOMEM);
  if (bh) {
    st->bh_kind = bh_walk_kind(M, p->bh_walk);
    st->bh_ntasks = bh_tasks(M, bh_chunks(M, st->tree->n_front, st->bh_kind),
                             bh_points_per_lane(st->bh_kind));
    if (dev_alloc_n(&st->bh_cost, st->bh_ntasks, s) ||
        dev_alloc_n(&st->bh_order, (size_t)st->bh_ntasks + TASK_ORDER_SCRATCH, s))
      return fail(FGA_ENOMEM);
    // the exact fixed-point force sums (zero; the epilogue leaves them zero)
    if (dev_alloc_n(&st->fb.acc, (size_t)3 * M, s)) return fail(FGA_ENOMEM);
    FGA_CUDA_TRY(cudaMemsetAsync(st->fb.acc, 0, sizeof(long long) * 3 * M, s));
  } else if (dev_alloc_n(&st->fb.hi, (size_t)st->fb.S * M, s) ||
             dev_alloc_n(&st->fb.lo, (size_t)st->fb.S * M, s)) {
    return fail(FGA_ENOMEM);
  }
  if ((rc = pack_template(Yn, mY, p->dt, M, bh, st->Y0, st->perm, s))) return fail(rc);
  if (dev_alloc_n(&st->partials, (size_t)epilogue_blocks(M) * NRED, s)) return fail(FGA_ENOMEM);
  st->max_traj = std::max(p->max_iter, 1);
  if (dev_alloc_n(&st->traj, (size_t)12 * st->max_traj, s)) return fail(FGA_ENOMEM);
  FGA_CUDA_TRY(cudaMemsetAsync(st->V, 0, sizeof(float4) * M, s));
  FGA_CUDA_TRY(cudaMemsetAsync(st->counter, 0, sizeof(unsigned), s));
  double* mu0 = nullptr;
  if (dev_alloc_n(&mu0, 3, s)) return fail(FGA_ENOMEM);
  if ((rc = centroid4(st->Y0, M, mu0, s))) return fail(rc);
  if ((rc = launch_state_init(st->ds, mu0, s))) return fail(rc);
  dev_free(mu0, s);
  *out = st;
  return FGA_OK;
}

static int step_launches(fga_state* st, int n_iter, cudaStream_t s);

// Without per-launch timing, n_iter >= FGA_STEP_GRAPH_MIN iterations are
// captured as one CUDA graph on a private stream ordered after `s` and
// launched once (no host round trip per launch; the GPU runs the loop's
// launches back to back). The graph, its stream and events are released by
// the runtime when the work completes, so the call stays asynchronous.
#ifndef FGA_STEP_GRAPH_MIN
#define FGA_STEP_GRAPH_MIN 4
#endif
// The executable graph of the calling thread's last capture, kept so that the
// next registration of the same shape (the same launches with other
// pointers) updates it in place instead of instantiating a new one. It is
// reused only once its last launch has completed (`done` has fired) and on
// the device it was made on.
struct StepGraphCache {
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t done = nullptr;
  int device = -1;
  ~StepGraphCache() {
    // the process may be ending with the runtime torn down: no CUDA calls here
  }
};
static thread_local StepGraphCache t_step_graph;

static EpiParams epi_params(const fga_state* st) {
  const fga_params& p = st->p;
  EpiParams ep{p.G, p.dt, p.eta, p.velocity_mode, (double)p.conv_tol, st->max_traj,
               1.0 / (double)st->M, 1.0 / (double)p.dt};
  ep.dim = p.dim;
  return ep;
}

// A small all-pairs pair: all n_iter iterations in one cluster launch, the
// same results as step_launches.
static int step_small(fga_state* st, int n_iter, cudaStream_t s) {
  const int traj_iters = std::max(0, st->max_traj - st->queued);
  const int rc = launch_small_loop(st->X4, st->N, st->Y0, st->M, st->ds, st->p.eps, st->plan, st->fb, st->V,
                                   st->partials, st->traj, traj_iters, epi_params(st),
                                   (unsigned long long)(st->N * st->M), n_iter, s);
  if (rc) return rc;
  st->queued += n_iter;
  return FGA_OK;
}

static int step_impl(fga_state* st, int n_iter, cudaStream_t s) {
  if (st->small_loop && !st->p.profile && st->p.method != FGA_BH) return step_small(st, n_iter, s);
  if (st->p.profile || n_iter < FGA_STEP_GRAPH_MIN) return step_launches(st, n_iter, s);
  cudaStream_t cs = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  struct Release {
    cudaStream_t& cs;
    cudaEvent_t& a;
    cudaEvent_t& b;
    cudaGraph_t& g;
    cudaGraphExec_t& e;
    ~Release() {
      if (e) cudaGraphExecDestroy(e);
      if (g) cudaGraphDestroy(g);
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
      if (cs) cudaStreamDestroy(cs);
    }
  } release{cs, ev_in, ev_out, graph, exec};
  FGA_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  FGA_CUDA_TRY(cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming));
  FGA_CUDA_TRY(cudaEventCreateWithFlags(&ev_out, cudaEventDisableTiming));
  FGA_CUDA_TRY(cudaEventRecord(ev_in, s));
  FGA_CUDA_TRY(cudaStreamWaitEvent(cs, ev_in, 0));
  FGA_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  const int lrc = step_launches(st, n_iter, cs);
  const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
  if (lrc != FGA_OK || ce != cudaSuccess) {
    if (lrc == FGA_OK)
      set_error(std::string("fga_step: graph capture failed: ") + cudaGetErrorString(ce));
    return lrc != FGA_OK ? lrc : FGA_ECUDA;
  }
  StepGraphCache& cache = t_step_graph;
  if (cache.exec && (cache.device != st->device || cudaEventQuery(cache.done) != cudaSuccess)) {
    // still running (or on another device): leave it to the runtime
    cudaGetLastError();
    cudaGraphExecDestroy(cache.exec);
    cudaEventDestroy(cache.done);
    cache.exec = nullptr;
    cache.done = nullptr;
  }
  if (cache.exec) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(cache.exec, graph, &info) == cudaSuccess) {
      exec = cache.exec;  // updated in place
    } else {
      cudaGetLastError();
      cudaGraphExecDestroy(cache.exec);
      cudaEventDestroy(cache.done);
    }
    cache.exec = nullptr;
    cache.done = nullptr;
  }
  if (!exec) FGA_CUDA_TRY(cudaGraphInstantiate(&exec, graph, 0));
  FGA_CUDA_TRY(cudaGraphLaunch(exec, cs));
  FGA_CUDA_TRY(cudaEventRecord(ev_out, cs));
  FGA_CUDA_TRY(cudaStreamWaitEvent(s, ev_out, 0));
  // keep the executable graph for the next call of this thread
  cache.exec = exec;
  cache.done = ev_out;
  cache.device = st->device;
  exec = nullptr;
  ev_out = nullptr;
  return FGA_OK;
}

static int step_launches(fga_state* st, int n_iter, cudaStream_t s) {
  const fga_params& p = st->p;
  const EpiParams ep = epi_params(st);
  const unsigned long long inter = p.method == FGA_BH ? 0ull : (unsigned long long)(st->N * st->M);
  if (p.profile) {
    const size_t need = 2 * (size_t)(st->timed + n_iter);
    while (st->events.size() < need) {
      cudaEvent_t e;
      FGA_CUDA_TRY(cudaEventCreate(&e));
      st->events.push_back(e);
    }
  }
  for (int k = 0; k < n_iter; ++k) {
    int rc;
    if (p.profile) FGA_CUDA_TRY(cudaEventRecord(st->events[2 * st->timed], s));
    if (p.method == FGA_BH) {
      rc = launch_bh(st->tree, st->Y0, st->M, st->ds, p.eps, p.theta, st->fb, s, st->bh_kind,
                     st->bh_have_order ? st->bh_order : nullptr, st->bh_cost);
      // heavy-first order for the following launches, refreshed on a schedule
      // (the task costs drift slowly as the template moves)
      ++st->bh_launches;
      if (rc == FGA_OK && bh_reorder_due(st->bh_launches)) {
        rc = launch_task_order(st->bh_cost, st->bh_ntasks, st->bh_order, s);
        st->bh_have_order = true;
      }
    } else {
      rc = launch_direct(st->X4, st->N, st->Y0, st->M, st->ds, p.eps, st->plan, st->fb, s);
    }
    if (rc) return rc;
    if (p.profile) {
      FGA_CUDA_TRY(cudaEventRecord(st->events[2 * st->timed + 1], s));
      ++st->timed;
    }
    if ((rc = launch_epilogue(st->Y0, st->M, st->fb, st->V, st->ds, st->partials, st->counter,
                              st->queued < st->max_traj ? st->traj : nullptr, ep, s, inter)))
      return rc;
    ++st->queued;
  }
  return FGA_OK;
}

extern "C" {

int fga_state_create(const float* Xn, const float* mX, int64_t N, const float* Yn, const float* mY,
                     int64_t M, const fga_tree* tree, const fga_params* p, fga_state** out,
                     void* stream) {
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  if (!out || !Xn || !Yn || N <= 0 || M <= 0 || N > (int64_t)1 << 30 || M > (int64_t)1 << 30) {
    set_error("fga_state_create: bad arguments");
    return FGA_EINVAL;
  }
  *out = nullptr;
  int rc = check_params(p, p && p->method != FGA_DIRECT && !tree);
  if (rc) return rc;
  fga_params resolved = *p;
  resolved.method = resolve_method(p, N);
  p = &resolved;
  Scratch sc(s);
  int* flags = nullptr;
  if (sc.alloc(&flags, 4)) return FGA_ENOMEM;
  FGA_CUDA_TRY(cudaMemsetAsync(flags, 0, 4 * sizeof(int), s));
  rc = check_finite(Xn, 3 * N, flags, s);
  if (!rc) rc = check_finite(Yn, 3 * M, flags + 1, s);
  if (!rc && mX) rc = check_masses(mX, N, flags + 2, s);
  if (!rc && mY) rc = check_masses(mY, M, flags + 3, s);
  if (rc) return rc;
  int h[4];
  if ((rc = read_flags(flags, 4, h, s))) return rc;
  if (h[0] || h[1] || h[2] || h[3]) {
    set_error("fga_state_create: non-finite coordinate or negative/non-finite mass");
    return FGA_EINVAL;
  }
  return state_create_checked(Xn, mX, N, Yn, mY, M, tree, p, out, s);
}

int fga_step(fga_state* st, int n_iter, void* stream) {
  clear_error();
  if (!st || n_iter < 0) {
    set_error("fga_step: bad arguments");
    return FGA_EINVAL;
  }
  return step_impl(st, n_iter, (cudaStream_t)stream);
}

int fga_state_get(fga_state* st, double R[9], double t[3], fga_stats* stats, void* stream) {
  clear_error();
  if (!st) {
    set_error("fga_state_get: null state");
    return FGA_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  DevState h;
  FGA_CUDA_TRY(cudaMemcpyAsync(&h, st->ds, sizeof(h), cudaMemcpyDeviceToHost, s));
  FGA_CUDA_TRY(cudaStreamSynchronize(s));
  if (R) std::memcpy(R, h.R, sizeof(h.R));
  if (t) std::memcpy(t, h.t, sizeof(h.t));
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->iterations = h.iter;
    stats->converged = h.converged;
    stats->degenerate_fits = h.degenerate;
    stats->interactions = (int64_t)h.interactions;
    stats->last_conv = h.last_conv;
    for (int k = 0; k < 3; ++k) {
      stats->net_force[k] = h.netF[k];
      stats->torque[k] = h.torque[k];
      stats->t_norm[k] = h.t[k];
    }
    std::memcpy(stats->R_norm, h.R, sizeof(h.R));
    double ms = 0;
    for (int k = 0; k < st->timed; ++k) {
      float e = 0.f;
      FGA_CUDA_TRY(cudaEventElapsedTime(&e, st->events[2 * k], st->events[2 * k + 1]));
      ms += e;
    }
    stats->force_ms = ms;
    stats->force_launches = st->timed;
  }
  int code = FGA_OK;
  if (h.status) {
    set_error("device check failed: non-finite transform");
    code = FGA_EINTERNAL;
  } else if (h.degenerate) {
    set_error("rank-deficient rigid fit in at least one iteration");
    code = FGA_EDEGENERATE;
  }
  if (stats) stats->status = code;
  return code;
}

int fga_state_trajectory(fga_state* st, double* out, int n, void* stream) {
  clear_error();
  if (!st || !out || n < 0) {
    set_error("fga_state_trajectory: bad arguments");
    return FGA_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int iters = 0;
  FGA_CUDA_TRY(cudaMemcpyAsync(&iters, &st->ds->iter, sizeof(int), cudaMemcpyDeviceToHost, s));
  FGA_CUDA_TRY(cudaStreamSynchronize(s));
  const int rows = std::min(std::min(n, iters), st->max_traj);
  if (rows > 0) {
    FGA_CUDA_TRY(cudaMemcpyAsync(out, st->traj, sizeof(double) * 12 * rows, cudaMemcpyDeviceToHost, s));
    FGA_CUDA_TRY(cudaStreamSynchronize(s));
  }
  return rows;
}

void fga_state_destroy(fga_state* st) {
  if (!st) return;
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != st->device) cudaSetDevice(st->device);
  cudaStream_t s = st->stream;
  dev_free(st->X4, s);
  dev_free(st->Y0, s);
  dev_free(st->perm, s);
  dev_free(st->V, s);
  dev_free(st->fb.hi, s);
  dev_free(st->fb.lo, s);
  dev_free(st->ds, s);
  dev_free(st->partials, s);
  dev_free(st->counter, s);
  dev_free(st->traj, s);
  dev_free(st->bh_cost, s);
  dev_free(st->bh_order, s);
  dev_free(st->fb.acc, s);
  if (st->own_tree) fga_tree_destroy(st->own_tree);
  for (cudaEvent_t e : st->events) cudaEventDestroy(e);
  if (prev != st->device) cudaSetDevice(prev);
  delete st;
}

int fga_register(const float* X, int64_t N, const float* Y, int64_t M, const float* mX,
                 const float* mY, const fga_params* p, double R_out[9], double t_out[3],
                 fga_stats* stats, void* stream) {
  clear_error();
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = (cudaStream_t)stream;
  if (!X || !Y || N <= 0 || M <= 0 || !R_out || !t_out || N > (int64_t)1 << 30 || M > (int64_t)1 << 30) {
    set_error("fga_register: bad arguments");
    return FGA_EINVAL;
  }
  int rc = check_register_params(p);
  if (rc) return rc;
  fga_params resolved = *p;
  resolved.method = resolve_method(p, N);
  p = &resolved;
  Scratch sc(s);
  int64_t h2d = 0, d2h = 0;
  Prepared pr;
  if ((rc = prepare_inputs(sc, X, N, Y, M, mX, mY, p, pr, h2d, s))) return rc;
  float *Xn = pr.Xn, *Yn = pr.Yn, *mXn = pr.mXn, *mYn = pr.mYn;
  double* info = pr.info;
  int* flags = pr.flags;
  fga_state* st = nullptr;
  if ((rc = state_create_checked(Xn, mXn, N, Yn, mYn, M, nullptr, p, &st, s))) return rc;
  rc = step_impl(st, p->max_iter, s);
  double h_info[8];
  int h_flags[8];
  if (!rc) {
    FGA_CUDA_TRY(cudaMemcpyAsync(h_info, info, sizeof(h_info), cudaMemcpyDeviceToHost, s));
    rc = read_flags(flags, 8, h_flags, s);
    d2h += sizeof(h_info) + sizeof(h_flags) + sizeof(DevState);
  }
  fga_stats local;
  int code = rc;
  double Rn[9], tn[3];
  if (!rc) code = fga_state_get(st, Rn, tn, &local, s);
  fga_state_destroy(st);
  if (rc) return rc;
  if (h_flags[0] || h_flags[1] || h_flags[2] || h_flags[3]) {
    set_error("fga_register: non-finite coordinate or negative/non-finite mass");
    return FGA_EINVAL;
  }
  if (!h_flags[4]) {
    set_error("fga_register: degenerate input (all centred coordinates equal)");
    return FGA_EINVAL;
  }
  std::memcpy(R_out, Rn, sizeof(Rn));
  if (p->normalize)
    fga_denormalize(Rn, tn, h_info, p->a, t_out);
  else
    std::memcpy(t_out, tn, sizeof(tn));
  if (stats) {
    *stats = local;
    std::memcpy(stats->norm_info, h_info, sizeof(h_info));
    stats->status = code;
    stats->h2d_bytes = h2d;
    stats->d2h_bytes = d2h;
    stats->elapsed_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return code;
}

}  // extern "C"
