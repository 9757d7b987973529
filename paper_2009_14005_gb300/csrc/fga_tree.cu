// Barnes-Hut tree of Algorithm 1 (Sec. IV-E) built on the GPU.
//
// Algorithm 1 splits the tight bounding box of X recursively at box midpoints
// down to depth max_depth. With max_depth bits per axis, the integer cell of a
// point along an axis, floor((x - lo)/(hi - lo) 2^bits), holds exactly the
// sequence of upper/lower decisions of those midpoint splits, so interleaving
// the three axes (Morton order) gives every point the path of Algorithm 1 as
// one 3*max_depth-bit key. After sorting the keys:
//   * a leaf of the tree is a run of equal keys (one point, or several points
//     that share a depth-max_depth cell);
//   * a cell that splits (>= 2 non-empty children) is a key range whose first
//     and last keys share exactly 3k leading bits: the cell sits at depth k and
//     its children are the sub-ranges with equal octant bits at level k + 1.
// Cells with a single non-empty child are not stored: their mass, CoM and
// point set equal the child's, and the child's smaller l makes BHForce give the
// same result without them.
//
// The build runs top-down one level per launch (children of a cell are stored
// contiguously, in octant order) and then bottom-up one level per launch for
// mass and centre of mass (FP64 sums, rounded once to FP32).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "fga_internal.cuh"

namespace fga {

static constexpr int TB = 256;

struct __align__(32) Sum4 {
  double x, y, z, w;
};

__global__ void k_gather_bodies(const float* __restrict__ X, const float* __restrict__ mX,
                                int64_t N, const int* __restrict__ idx, float4* __restrict__ bodies,
                                int* __restrict__ body_index) {
  const float m_default = (float)(1.0 / (double)N);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int j = idx[i];
    bodies[i] = make_float4(X[3 * (int64_t)j], X[3 * (int64_t)j + 1], X[3 * (int64_t)j + 2],
                            mX ? mX[j] : m_default);
    body_index[i] = j;
  }
}

__global__ void k_head_flags(const unsigned long long* __restrict__ keys, int64_t N,
                             unsigned* __restrict__ flags) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    flags[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
}

// ustart[u] = first sorted body of unique key u; ukey[u] = the key; ustart[n_u] = N.
__global__ void k_unique(const unsigned long long* __restrict__ keys, int64_t N,
                         const unsigned* __restrict__ flags, const unsigned* __restrict__ uid,
                         const unsigned* __restrict__ n_unique, unsigned long long* __restrict__ ukey,
                         int* __restrict__ ustart) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (flags[i]) {
      ustart[uid[i]] = (int)i;
      ukey[uid[i]] = keys[i];
    }
    if (i == 0) ustart[*n_unique] = (int)N;
  }
}

struct LevelInfo {
  int start[32];
  int count[32];
  int overflow;
};

__global__ void k_tree_init(const unsigned* __restrict__ n_unique, LevelInfo* lv,
                            int2* __restrict__ node_range, int4* __restrict__ node_info) {
  for (int i = 0; i < 32; ++i) {
    lv->start[i] = 0;
    lv->count[i] = 0;
  }
  lv->count[0] = 1;
  lv->overflow = 0;
  node_range[0] = make_int2(0, (int)*n_unique);
  node_info[0] = make_int4(0, 0, 0, 0);  // w: depth hint of the root
}

__device__ __forceinline__ int octant_of(unsigned long long key, int shift) {
  return (int)((key >> shift) & 7ull);
}

// One level of the top-down build. Node v of level L covers unique keys
// [us, ue). A single key is a leaf; otherwise the cell depth is the common
// prefix length of its first and last key divided by 3, and the children are
// the runs of equal octant at the next level, found by binary search.
__global__ void k_build_level(int L, int D, int cap, const unsigned long long* __restrict__ ukey,
                              const int* __restrict__ ustart, LevelInfo* lv,
                              int2* __restrict__ node_range, int4* __restrict__ node_info,
                              int2* __restrict__ node_bodies, double ext2) {
  if (lv->overflow) return;  // capacity guard fired on an earlier level
  const int start = lv->start[L], cnt = lv->count[L];
  const int next_start = start + cnt;
  if (blockIdx.x == 0 && threadIdx.x == 0) lv->start[L + 1] = next_start;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x) {
    const int v = start + t;
    const int2 r = node_range[v];
    const int us = r.x, ue = r.y;
    const int b0 = ustart[us], b1 = ustart[ue];
    node_bodies[v] = make_int2(b0, b1);
    if (ue - us == 1) {
      const int nb = b1 - b0;
      const int depth = nb > 1 ? D : node_info[v].w;
      const float l2 = nb > 1 ? (float)ldexp(ext2, -2 * D) : 0.0f;
      node_info[v] = make_int4(__float_as_int(l2), b0, -nb, depth);
      continue;
    }
    const unsigned long long k1 = ukey[us], k2 = ukey[ue - 1];
    const int delta = __clzll((long long)(k1 ^ k2)) - (64 - 3 * D);
    const int depth = delta / 3;
    const int shift = 3 * (D - depth - 1);
    int bnd[9];
    bnd[0] = us;
    bnd[8] = ue;
    for (int o = 1; o < 8; ++o) {
      int lo = bnd[o - 1], hi = ue;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (octant_of(ukey[mid], shift) < o) lo = mid + 1; else hi = mid;
      }
      bnd[o] = lo;
    }
    int nc = 0;
    for (int o = 0; o < 8; ++o) nc += bnd[o + 1] > bnd[o];
    const int base = atomicAdd(&lv->count[L + 1], nc);
    const int first = next_start + base;
    if (first + nc > cap) {
      atomicExch(&lv->overflow, 1);
      continue;
    }
    int c = 0;
    for (int o = 0; o < 8; ++o)
      if (bnd[o + 1] > bnd[o]) {
        node_range[first + c] = make_int2(bnd[o], bnd[o + 1]);
        node_info[first + c] = make_int4(0, 0, 0, depth + 1);  // depth hint for singleton leaves
        ++c;
      }
    node_info[v] = make_int4(__float_as_int((float)ldexp(ext2, -2 * depth)), first, nc, depth);
  }
}

// Bottom-up: FP64 sums of mass and mass-weighted position (and plain position
// sums for massless cells) from bodies (leaves) or children (internal cells),
// and the number of pre-order records of each subtree (a leaf with nb >= 2
// particles takes 1 + nb records, see k_interleave_pre).
__global__ void k_mass_level(int L, const LevelInfo* __restrict__ lv, const float4* __restrict__ bodies,
                             const int4* __restrict__ node_info, Sum4* __restrict__ sum_m,
                             Sum4* __restrict__ sum_p, float4* __restrict__ node_cm,
                             int* __restrict__ node_size) {
  if (lv->overflow) return;
  const int start = lv->start[L], cnt = lv->count[L];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x) {
    const int v = start + t;
    const int4 inf = node_info[v];
    Sum4 a = {0, 0, 0, 0}, p = {0, 0, 0, 0};
    int size = 1;
    if (inf.z < 0) {
      size = inf.z < -1 ? 1 - inf.z : 1;
      for (int b = inf.y; b < inf.y - inf.z; ++b) {
        const float4 q = bodies[b];
        a.x += (double)q.w * q.x;
        a.y += (double)q.w * q.y;
        a.z += (double)q.w * q.z;
        a.w += q.w;
        p.x += q.x;
        p.y += q.y;
        p.z += q.z;
        p.w += 1.0;
      }
    } else {
      for (int c = inf.y; c < inf.y + inf.z; ++c) {
        const Sum4 ca = sum_m[c], cp = sum_p[c];
        a.x += ca.x; a.y += ca.y; a.z += ca.z; a.w += ca.w;
        p.x += cp.x; p.y += cp.y; p.z += cp.z; p.w += cp.w;
        size += node_size[c];
      }
    }
    node_size[v] = size;
    sum_m[v] = a;
    sum_p[v] = p;
    node_cm[v] = a.w > 0 ? make_float4((float)(a.x / a.w), (float)(a.y / a.w), (float)(a.z / a.w), (float)a.w)
                         : make_float4((float)(p.x / p.w), (float)(p.y / p.w), (float)(p.z / p.w), 0.0f);
  }
}

// Top-down: depth-first pre-order record index of every cell. A cell's first
// child follows it directly; each further child follows its previous
// sibling's subtree. pos[0] = 0 (the root) is set before the first level.
__global__ void k_preorder_level(int L, const LevelInfo* __restrict__ lv, const int4* __restrict__ node_info,
                                 const int* __restrict__ node_size, int* __restrict__ node_pos) {
  if (lv->overflow) return;
  const int start = lv->start[L], cnt = lv->count[L];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x) {
    const int v = start + t;
    const int4 inf = node_info[v];
    if (inf.z <= 0) continue;
    int run = node_pos[v] + 1;
    for (int c = inf.y; c < inf.y + inf.z; ++c) {
      node_pos[c] = run;
      run += node_size[c];
    }
  }
}

// Frontier for splitting BH work (see FrontCell): starting from the root,
// repeatedly replace the frontier cell holding the most bodies by its
// children, until about `target` cells (never more) or only
// leaves remain. Uses the first levels of the breadth-first node arrays.
static int build_frontier(fga_tree* T, int target, const int* d_pos, const int* d_size, cudaStream_t s) {
  const int64_t P = std::min<int64_t>(T->n_nodes, 1 << 16);
  std::vector<int4> info(P);
  std::vector<int2> nb(P);
  std::vector<int> pos(P), size(P);
  FGA_CUDA_TRY(cudaMemcpyAsync(info.data(), T->node_info, sizeof(int4) * P, cudaMemcpyDeviceToHost, s));
  FGA_CUDA_TRY(cudaMemcpyAsync(nb.data(), T->node_bodies, sizeof(int2) * P, cudaMemcpyDeviceToHost, s));
  FGA_CUDA_TRY(cudaMemcpyAsync(pos.data(), d_pos, sizeof(int) * P, cudaMemcpyDeviceToHost, s));
  FGA_CUDA_TRY(cudaMemcpyAsync(size.data(), d_size, sizeof(int) * P, cudaMemcpyDeviceToHost, s));
  float4 root;
  FGA_CUDA_TRY(cudaMemcpyAsync(&root, T->node_cm, sizeof(float4), cudaMemcpyDeviceToHost, s));
  FGA_CUDA_TRY(cudaStreamSynchronize(s));
  T->mass_total = (double)root.w;
  struct Item {
    int node;
    std::vector<int> path;
  };
  std::vector<Item> front{{0, {}}};
  const int kMax = std::max(1, target);
  while ((int)front.size() < kMax) {
    int best = -1, best_n = 1;
    for (int k = 0; k < (int)front.size(); ++k) {
      const int v = front[k].node;
      const int4 in = info[v];
      if (in.z <= 0 || (int64_t)in.y + in.z > P || (int)front[k].path.size() >= FRONT_MAX_PATH) continue;
      const int n = nb[v].y - nb[v].x;
      if (n > best_n) {
        best_n = n;
        best = k;
      }
    }
    if (best < 0) break;
    const int v = front[best].node;
    if ((int)front.size() - 1 + info[v].z > kMax) break;
    std::vector<int> path = front[best].path;
    path.push_back(v);
    front.erase(front.begin() + best);
    for (int c = 0; c < info[v].z; ++c) front.push_back({info[v].y + c, path});
  }
  std::sort(front.begin(), front.end(),
            [&](const Item& a, const Item& b) { return nb[a.node].x < nb[b.node].x; });
  // in depth-first record indices (pos, size: pre-order index and record count
  // of each cell's subtree)
  std::vector<FrontCell> table(front.size());
  for (size_t k = 0; k < front.size(); ++k) {
    FrontCell& fc = table[k];
    std::memset(&fc, 0, sizeof(fc));
    const int v = front[k].node;
    fc.node = pos[v];
    fc.end = pos[v] + size[v];
    fc.npath = (int)front[k].path.size();
    for (int j = 0; j < fc.npath; ++j) {
      const int a = front[k].path[j];
      fc.path[j] = pos[a];
      if (nb[v].x == nb[a].x) fc.first_mask |= 1u << j;
    }
  }
  int rc = dev_alloc_n(&T->front, table.size(), s);
  if (rc) return rc;
  FGA_CUDA_TRY(cudaMemcpyAsync(T->front, table.data(), sizeof(FrontCell) * table.size(),
                               cudaMemcpyHostToDevice, s));
  FGA_CUDA_TRY(cudaStreamSynchronize(s));
  T->n_front = (int)table.size();
  return FGA_OK;
}

// The depth-first records: cell v is record pos[v], with CoM and mass in
// pcm, (l^2, subtree size) in pls and (count, first body) in pcf. A
// single-particle leaf gets l^2 = -1 (always accepted: its one exact term). A
// leaf holding nb >= 2 particles keeps its l^2 (its monopole when accepted)
// and is followed by nb single-particle records, one per particle in order,
// which the walk enters when the leaf is rejected: the same exact terms as
// the leaf's particle loop of Algorithm 2.
__global__ void k_interleave_pre(const float4* __restrict__ cm, const int4* __restrict__ info,
                                 const int* __restrict__ size, const int* __restrict__ pos,
                                 const float4* __restrict__ bodies, int64_t n, float4* __restrict__ pcm,
                                 float2* __restrict__ pls, int2* __restrict__ pcf) {
  const float2 single_ls = make_float2(-1.0f, __int_as_float(1));
  const int2 single_cf = make_int2(-1, 0);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int4 in = info[i];
    const int64_t p = pos[i];
    pcm[p] = cm[i];
    if (in.z == -1) {
      pls[p] = single_ls;
      pcf[p] = single_cf;
      continue;
    }
    pls[p] = make_float2(__int_as_float(in.x), __int_as_float(size[i]));
    pcf[p] = make_int2(in.z, in.z < 0 ? in.y : 0);
    for (int b = 0; b < -in.z; ++b) {
      pcm[p + 1 + b] = bodies[in.y + b];
      pls[p + 1 + b] = single_ls;
      pcf[p + 1 + b] = single_cf;
    }
  }
}

// On every way out of tree_build: frees the build's scratch (stream-ordered)
// and, unless the build succeeded, the tree itself.
struct BuildGuard {
  cudaStream_t s;
  fga_tree* tree;
  std::vector<void*> bufs;
  void add(void* p) { bufs.push_back(p); }
  void release(void* p) {
    for (void*& b : bufs)
      if (b == p) {
        dev_free(b, s);
        b = nullptr;
      }
  }
  ~BuildGuard() {
    for (void* b : bufs) dev_free(b, s);
    if (tree) fga_tree_destroy(tree);
  }
};

int tree_build(const float* X, const float* mX, int64_t N, int D, fga_tree** out, cudaStream_t s,
               int front_target) {
  if (N > ((int64_t)1 << 26)) {
    set_error("tree_build: at most 2^26 points per tree");
    return FGA_EINVAL;
  }
  fga_tree* T = new fga_tree();
  T->N = N;
  T->max_depth = D;
  T->stream = s;
  cudaGetDevice(&T->device);
  BuildGuard guard{s, T, {}};
  const int64_t cap = 2 * N;
  int rc = 0;
  rc |= dev_alloc_n(&T->bodies, N, s);
  rc |= dev_alloc_n(&T->body_index, N, s);
  rc |= dev_alloc_n(&T->keys, N, s);
  rc |= dev_alloc_n(&T->node_cm, cap, s);
  rc |= dev_alloc_n(&T->node_info, cap, s);
  rc |= dev_alloc_n(&T->node_bodies, cap, s);
  // build scratch
  unsigned long long *ktmp = nullptr, *ukey = nullptr;
  int *idx = nullptr, *itmp = nullptr, *ustart = nullptr;
  unsigned *flags = nullptr, *uid = nullptr, *n_u = nullptr;
  int2* node_range = nullptr;
  int *node_size = nullptr, *node_pos = nullptr;
  Sum4 *sum_m = nullptr, *sum_p = nullptr;
  float* box = nullptr;
  LevelInfo* lv = nullptr;
  rc |= dev_alloc_n(&ktmp, N, s);
  rc |= dev_alloc_n(&ukey, N, s);
  rc |= dev_alloc_n(&idx, N, s);
  rc |= dev_alloc_n(&itmp, N, s);
  rc |= dev_alloc_n(&ustart, N + 1, s);
  rc |= dev_alloc_n(&flags, N, s);
  rc |= dev_alloc_n(&uid, N, s);
  rc |= dev_alloc_n(&n_u, 1, s);
  rc |= dev_alloc_n(&node_range, cap, s);
  rc |= dev_alloc_n(&node_size, cap, s);
  rc |= dev_alloc_n(&node_pos, cap, s);
  rc |= dev_alloc_n(&sum_m, cap, s);
  rc |= dev_alloc_n(&sum_p, cap, s);
  rc |= dev_alloc_n(&box, 6, s);
  rc |= dev_alloc_n(&lv, 1, s);
  for (void* b : {(void*)ktmp, (void*)ukey, (void*)idx, (void*)itmp, (void*)ustart, (void*)flags, (void*)uid,
                  (void*)n_u, (void*)node_range, (void*)node_size, (void*)node_pos, (void*)sum_m, (void*)sum_p,
                  (void*)box, (void*)lv})
    guard.add(b);
  if (rc) return FGA_ENOMEM;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((N + TB - 1) / TB, 8 * sm_count()));
  if ((rc = bbox_xyz(X, N, box, box + 3, s))) return rc;
  if ((rc = morton_keys(X, N, box, box + 3, D, T->keys, idx, s))) return rc;
  if ((rc = radix_sort_pairs(T->keys, idx, ktmp, itmp, N, 3 * D, s))) return rc;
  k_gather_bodies<<<grid, TB, 0, s>>>(X, mX, N, idx, T->bodies, T->body_index);
  FGA_LAUNCH_CHECK("gather_bodies");
  k_head_flags<<<grid, TB, 0, s>>>(T->keys, N, flags);
  FGA_LAUNCH_CHECK("head_flags");
  if ((rc = scan_exclusive(flags, uid, N, n_u, s))) return rc;
  k_unique<<<grid, TB, 0, s>>>(T->keys, N, flags, uid, n_u, ukey, ustart);
  FGA_LAUNCH_CHECK("unique");
  k_tree_init<<<1, 1, 0, s>>>(n_u, lv, node_range, T->node_info);
  FGA_LAUNCH_CHECK("tree_init");
  float lo[3], hi[3];
  FGA_CUDA_TRY(cudaMemcpyAsync(lo, box, sizeof(lo), cudaMemcpyDeviceToHost, s));
  FGA_CUDA_TRY(cudaMemcpyAsync(hi, box + 3, sizeof(hi), cudaMemcpyDeviceToHost, s));
  FGA_CUDA_TRY(cudaStreamSynchronize(s));
  double ext2 = 0;
  for (int k = 0; k < 3; ++k) {
    T->box_lo[k] = lo[k];
    T->box_hi[k] = hi[k];
    const double e = (double)hi[k] - (double)lo[k];
    ext2 += e * e;
  }
  for (int L = 0; L <= D; ++L) {
    k_build_level<<<grid, TB, 0, s>>>(L, D, (int)cap, ukey, ustart, lv, node_range, T->node_info,
                                      T->node_bodies, ext2);
    FGA_LAUNCH_CHECK("build_level");
  }
  for (int L = D; L >= 0; --L) {
    k_mass_level<<<grid, TB, 0, s>>>(L, lv, T->bodies, T->node_info, sum_m, sum_p, T->node_cm, node_size);
    FGA_LAUNCH_CHECK("mass_level");
  }
  FGA_CUDA_TRY(cudaMemsetAsync(node_pos, 0, sizeof(int), s));
  for (int L = 0; L <= D; ++L) {
    k_preorder_level<<<grid, TB, 0, s>>>(L, lv, T->node_info, node_size, node_pos);
    FGA_LAUNCH_CHECK("preorder_level");
  }
  LevelInfo h_lv;
  unsigned h_nu = 0;
  int h_npre = 0;
  FGA_CUDA_TRY(cudaMemcpyAsync(&h_lv, lv, sizeof(h_lv), cudaMemcpyDeviceToHost, s));
  FGA_CUDA_TRY(cudaMemcpyAsync(&h_nu, n_u, sizeof(h_nu), cudaMemcpyDeviceToHost, s));
  FGA_CUDA_TRY(cudaMemcpyAsync(&h_npre, node_size, sizeof(int), cudaMemcpyDeviceToHost, s));
  FGA_CUDA_TRY(cudaStreamSynchronize(s));
  // the scratch the remaining steps do not read (node_size, node_pos: below)
  for (void* b : {(void*)ktmp, (void*)ukey, (void*)idx, (void*)itmp, (void*)ustart, (void*)flags, (void*)uid,
                  (void*)n_u, (void*)node_range, (void*)sum_m, (void*)sum_p, (void*)box, (void*)lv})
    guard.release(b);
  if (h_lv.overflow) {
    set_error("tree_build: node capacity exceeded");
    return FGA_EINTERNAL;
  }
  T->n_nodes = h_lv.start[D + 1];
  T->n_unique = (int)h_nu;
  T->n_pre = h_npre;  // the root's subtree: every record
  if ((rc = build_frontier(T, front_target, node_pos, node_size, s))) return rc;
  if (dev_alloc_n(&T->node_pre, (size_t)2 * T->n_pre, s)) return FGA_ENOMEM;
  k_interleave_pre<<<grid, TB, 0, s>>>(T->node_cm, T->node_info, node_size, node_pos, T->bodies, T->n_nodes,
                                       T->node_pre, const_cast<float2*>(pre_ls(T)),
                                       const_cast<int2*>(pre_cf(T)));
  FGA_LAUNCH_CHECK("interleave_pre");
  guard.tree = nullptr;  // built: the caller owns it
  *out = T;
  return FGA_OK;
}

}  // namespace fga

using namespace fga;

extern "C" void fga_tree_destroy(fga_tree* t) {
  if (!t) return;
  int prev = 0;
  cudaGetDevice(&prev);
  if (prev != t->device) cudaSetDevice(t->device);
  dev_free(t->bodies, t->stream);
  dev_free(t->body_index, t->stream);
  dev_free(t->keys, t->stream);
  dev_free(t->node_cm, t->stream);
  dev_free(t->node_info, t->stream);
  dev_free(t->node_bodies, t->stream);
  dev_free(t->front, t->stream);
  dev_free(t->node_pre, t->stream);
  if (prev != t->device) cudaSetDevice(prev);
  delete t;
}

extern "C" int64_t fga_tree_node_count(const fga_tree* t) { return t ? t->n_nodes : 0; }

extern "C" int64_t fga_tree_preorder(const fga_tree* t, int64_t cap, float* out, void* stream) {
  clear_error();
  if (!t) {
    set_error("fga_tree_preorder: null tree");
    return FGA_EINVAL;
  }
  if (cap == 0) return t->n_pre;
  if (cap < t->n_pre || !out) {
    set_error("fga_tree_preorder: buffer smaller than the record count");
    return FGA_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  // the three record arrays, interleaved into 32-byte host records
  const size_t rec = 8 * sizeof(float);
  FGA_CUDA_TRY(cudaMemcpy2DAsync(out, rec, pre_cm(t), sizeof(float4), sizeof(float4), (size_t)t->n_pre,
                                 cudaMemcpyDeviceToHost, s));
  FGA_CUDA_TRY(cudaMemcpy2DAsync(out + 4, rec, pre_ls(t), sizeof(float2), sizeof(float2), (size_t)t->n_pre,
                                 cudaMemcpyDeviceToHost, s));
  FGA_CUDA_TRY(cudaMemcpy2DAsync(out + 6, rec, pre_cf(t), sizeof(int2), sizeof(int2), (size_t)t->n_pre,
                                 cudaMemcpyDeviceToHost, s));
  FGA_CUDA_TRY(cudaStreamSynchronize(s));
  return t->n_pre;
}

extern "C" int64_t fga_tree_export(const fga_tree* t, int64_t cap, int64_t* ints, double* dbls,
                                   int64_t* leaf_of, void* stream) {
  clear_error();
  if (!t) {
    set_error("fga_tree_export: null tree");
    return FGA_EINVAL;
  }
  if (cap == 0) return t->n_nodes;
  if (cap < t->n_nodes || !ints || !dbls) {
    set_error("fga_tree_export: buffers smaller than the node count");
    return FGA_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = t->n_nodes, N = t->N;
  std::vector<float4> cm(n);
  std::vector<int4> info(n);
  std::vector<int2> nb(n);
  std::vector<unsigned long long> keys(N);
  std::vector<int> bidx(N);
  FGA_CUDA_TRY(cudaMemcpyAsync(cm.data(), t->node_cm, sizeof(float4) * n, cudaMemcpyDeviceToHost, s));
  FGA_CUDA_TRY(cudaMemcpyAsync(info.data(), t->node_info, sizeof(int4) * n, cudaMemcpyDeviceToHost, s));
  FGA_CUDA_TRY(cudaMemcpyAsync(nb.data(), t->node_bodies, sizeof(int2) * n, cudaMemcpyDeviceToHost, s));
  FGA_CUDA_TRY(cudaMemcpyAsync(keys.data(), t->keys, sizeof(unsigned long long) * N,
                               cudaMemcpyDeviceToHost, s));
  FGA_CUDA_TRY(cudaMemcpyAsync(bidx.data(), t->body_index, sizeof(int) * N, cudaMemcpyDeviceToHost, s));
  FGA_CUDA_TRY(cudaStreamSynchronize(s));
  const int D = t->max_depth;
  double ext2 = 0;
  for (int k = 0; k < 3; ++k) {
    const double e = (double)t->box_hi[k] - (double)t->box_lo[k];
    ext2 += e * e;
  }
  const double root_l = std::sqrt(ext2);
  // iterative pre-order DFS, children in stored (octant) order
  std::vector<std::pair<int, int64_t>> stack;  // (node, parent export index)
  stack.push_back({0, -1});
  int64_t out_i = 0;
  while (!stack.empty()) {
    auto [v, parent] = stack.back();
    stack.pop_back();
    const int4 inf = info[v];
    const int depth = inf.w;
    const unsigned long long key = keys[nb[v].x];
    unsigned q[3] = {0, 0, 0};
    for (int bit = 0; bit < D; ++bit)
      for (int k = 0; k < 3; ++k) q[k] |= (unsigned)((key >> (3 * bit + k)) & 1ull) << bit;
    int64_t* I = ints + 7 * out_i;
    double* Dd = dbls + 5 * out_i;
    I[0] = depth;
    for (int k = 0; k < 3; ++k) I[1 + k] = (int64_t)(q[k] >> (D - depth));
    I[4] = nb[v].y - nb[v].x;
    I[5] = inf.z < 0;
    I[6] = parent;
    Dd[0] = cm[v].w;
    Dd[1] = cm[v].x;
    Dd[2] = cm[v].y;
    Dd[3] = cm[v].z;
    Dd[4] = std::ldexp(root_l, -depth);
    if (inf.z < 0 && leaf_of)
      for (int b = nb[v].x; b < nb[v].y; ++b) leaf_of[bidx[b]] = out_i;
    if (inf.z > 0)
      for (int c = inf.z - 1; c >= 0; --c) stack.push_back({inf.y + c, out_i});
    ++out_i;
  }
  return out_i;
}
