// Small all-pairs registrations in one launch: the whole iteration loop of
// Algorithm 2 (Eq. 6 forces, Eqs. 7-10 ODE step, Eq. 14 reductions and rigid
// fit, Eq. 16, composition and stop test) runs in one thread-block cluster.
//
// For a pair of a few thousand points an iteration is a few microseconds of
// arithmetic spread over a handful of SMs, and the separate force and
// epilogue launches spend most of the iteration on launch gaps, the
// last-block handshake and the copy of the state into and out of global
// memory. Here the cluster stays resident for all iterations:
//  - the reference points are staged in shared memory once, in every CTA;
//  - the force phase computes the same (template block, source split) items
//    as k_direct's blocks, with the same tiles in the same order, and leaves
//    the same compensated partial sums;
//  - the epilogue phase computes the same blocks of points as k_epilogue
//    (same points per thread, same block partials of the FP64 reductions);
//  - every CTA then adds the block partials and takes the rigid fit on its
//    own copy of the state in shared memory. All copies run the same code on
//    the same values, so they agree bit for bit and no CTA waits for another
//    to publish the transform; CTA 0 writes the trajectory and, at the end,
//    the state.
// Two cluster barriers per iteration order the phases: after the force phase
// (partial sums complete) and after the epilogue phase (block partials
// complete). A CTA can run ahead into the next force phase while another is
// still in its fit; the next writes of the block partials come only after
// the next first barrier, which that CTA reaches after its fit.
// Results are bit-identical to the separate launches of fga_force.cu.
#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>

#include "fga_device.cuh"
#include "fga_epi.cuh"

namespace cg = cooperative_groups;

namespace fga {

namespace {

constexpr int SL_NT = EPI_BS;  // threads per CTA (the epilogue's block size)
constexpr int SL_MAX_CTAS = 16;

// One block of k_direct<BS, QPT>: template points qb * BS * QPT + t + q * BS
// against the sources of split `split`, read from the staged copy xs (paired
// layout for even QPT, zero-padded to a multiple of BS). Writes the split's
// compensated sums (L2 stores: another CTA reads them).
template <int BS, int QPT>
__device__ __forceinline__ void direct_item(const float4* xs, int64_t N, int64_t chunk, int split, int64_t qb,
                                            int t, const float4* __restrict__ Y0, int64_t M, const Xf& xf,
                                            float eps2, float4* hi_out, float4* lo_out) {
  constexpr bool PAIRED = QPT % 2 == 0;
  const int64_t j0 = (int64_t)split * chunk;
  const int64_t j1 = min(N, j0 + chunk);
  float yx[QPT], yy[QPT], yz[QPT];
  float hx[QPT], hy[QPT], hz[QPT], lx[QPT], ly[QPT], lz[QPT];
  const int64_t qbase = qb * BS * QPT + t;
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
    float px[QPT], py[QPT], pz[QPT];
    if constexpr (PAIRED) {
      const float4* tile = xs + 2 * b;
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
      const float4* tile = xs + b;
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
  }
#pragma unroll
  for (int q = 0; q < QPT; ++q) {
    const int64_t i = qbase + (int64_t)q * BS;
    if (i < M) {
      __stcg(&hi_out[(int64_t)split * M + i], make_float4(hx[q], hy[q], hz[q], 0.f));
      __stcg(&lo_out[(int64_t)split * M + i], make_float4(lx[q], ly[q], lz[q], 0.f));
    }
  }
}

// epi_point over all S slots, with the slots read from L2 (other CTAs of
// the cluster wrote them in this launch): the same loads in the same order
// and the same compensated sum.
__device__ __forceinline__ void epi_point_l2(int64_t i, const float4* __restrict__ Y0, const float4* hi,
                                             const float4* lo, int S, int64_t M, float4* __restrict__ V,
                                             const EpiParams& ep, const EpiCtx& c, float (&r)[NRED]) {
  const float4 y0 = Y0[i];
  float ahx = 0.f, ahy = 0.f, ahz = 0.f, alx = 0.f, aly = 0.f, alz = 0.f;
  for (int s = 0; s < S; s += 4) {
    float4 h[4], l[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const bool ok = s + k < S;
      h[k] = ok ? __ldcg(&hi[(int64_t)(s + k) * M + i]) : make_float4(0.f, 0.f, 0.f, 0.f);
      l[k] = ok ? __ldcg(&lo[(int64_t)(s + k) * M + i]) : make_float4(0.f, 0.f, 0.f, 0.f);
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
  epi_ode(i, y0, ahx + alx, ahy + aly, ahz + alz, V, ep, c, r);
}

// The loop. Grid = one cluster of gridDim.x CTAs of SL_NT threads. The
// number of iterations each CTA runs depends only on its copy of the state,
// which is the same in every CTA, so all CTAs pass the same cluster barriers.
template <int BS, int QPT>
__global__ void __launch_bounds__(SL_NT, 1)
    k_small_loop(const float4* __restrict__ X, int64_t N, int64_t chunk, int S, const float4* __restrict__ Y0,
                 int64_t M, DevState* ds_g, float eps2, float4* hi, float4* lo, float4* __restrict__ V,
                 double* partials, int nblk_epi, double* traj, int traj_iters, EpiParams ep,
                 unsigned long long inter_add, int n_iter) {
  static_assert(SL_NT % BS == 0, "whole template blocks per CTA");
  constexpr bool PAIRED = QPT % 2 == 0;
  constexpr int SUB = SL_NT / BS;  // k_direct blocks computed at once per CTA
  constexpr int NW = (int)(sizeof(DevState) / sizeof(unsigned long long));
  static_assert(NW <= SL_NT, "one state word per thread");
  extern __shared__ float4 xs[];  // the sources: (x,x,y,y), (z,z,m,m) each if PAIRED, else (x,y,z,m)
  __shared__ DevState st;
  __shared__ double s_red[NRED];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int ncta = (int)cluster.num_blocks();

  const int64_t npad = (N + BS - 1) / BS * BS;
  for (int64_t j = threadIdx.x; j < npad; j += SL_NT) {
    const float4 src = j < N ? X[j] : make_float4(0.f, 0.f, 0.f, 0.f);  // m = 0 pads the tail
    if constexpr (PAIRED) {
      xs[2 * j] = make_float4(src.x, src.x, src.y, src.y);
      xs[2 * j + 1] = make_float4(src.z, src.z, src.w, src.w);
    } else {
      xs[j] = src;
    }
  }
  if (threadIdx.x < NW)
    reinterpret_cast<unsigned long long*>(&st)[threadIdx.x] =
        __ldcg(reinterpret_cast<const unsigned long long*>(ds_g) + threadIdx.x);
  __syncthreads();

  const int64_t qblocks = (M + (int64_t)BS * QPT - 1) / ((int64_t)BS * QPT);
  const int64_t items = qblocks * S;
  const int sub = threadIdx.x / BS, t = threadIdx.x % BS;
  for (int it = 0; it < n_iter; ++it) {
    if (st.done) break;
    {
      const Xf xf = load_xf(&st);
      for (int64_t w = (int64_t)rank * SUB + sub; w < items; w += (int64_t)ncta * SUB)
        direct_item<BS, QPT>(xs, N, chunk, (int)(w / qblocks), w % qblocks, t, Y0, M, xf, eps2, hi, lo);
    }
    cluster.sync();
    {
      const EpiCtx c = load_epi(&st);
      for (int b = rank; b < nblk_epi; b += ncta) {
        float r[NRED];
#pragma unroll
        for (int k = 0; k < NRED; ++k) r[k] = 0.f;
        for (int64_t i = (int64_t)b * SL_NT + threadIdx.x; i < M; i += (int64_t)nblk_epi * SL_NT)
          epi_point_l2(i, Y0, hi, lo, S, M, V, ep, c, r);
        epi_block_partial(r, partials + (int64_t)b * NRED);
        __syncthreads();
      }
    }
    cluster.sync();
    epi_last_reduce(partials, nblk_epi, s_red);
    rigid_step_smem(s_red, M, &st, ep, (rank == 0 && it < traj_iters) ? traj : nullptr, inter_add);
  }
  if (rank == 0 && threadIdx.x < NW)
    reinterpret_cast<unsigned long long*>(ds_g)[threadIdx.x] =
        reinterpret_cast<const unsigned long long*>(&st)[threadIdx.x];
}

using SmallKernel = void (*)(const float4*, int64_t, int64_t, int, const float4*, int64_t, DevState*, float,
                             float4*, float4*, float4*, double*, int, double*, int, EpiParams,
                             unsigned long long, int);

SmallKernel small_kernel(int bs, int qpt) {
  if (bs == 128 && qpt == 1) return k_small_loop<128, 1>;
  if (bs == 128 && qpt == 2) return k_small_loop<128, 2>;
  if (bs == 128 && qpt == 4) return k_small_loop<128, 4>;
  if (bs == 256 && qpt == 1) return k_small_loop<256, 1>;
  if (bs == 256 && qpt == 2) return k_small_loop<256, 2>;
  if (bs == 256 && qpt == 4) return k_small_loop<256, 4>;
  return nullptr;
}

size_t small_smem_bytes(int64_t N, int bs, int qpt) {
  const int64_t npad = (N + bs - 1) / bs * bs;
  return (size_t)npad * sizeof(float4) * (qpt % 2 == 0 ? 2 : 1);
}

// Per device (ordinals 0-7; others take the separate launches) and kernel:
// the attributes are set once, and the largest cluster (16, else 8) that the
// device can hold at this kernel's shared memory size is found once (0: none).
struct SmallSetup {
  std::mutex mu;
  int max_cluster[8][6] = {};  // [device][tile shape], -1 unknown
  SmallSetup() {
    for (auto& d : max_cluster)
      for (int& v : d) v = -1;
  }
};
SmallSetup& small_setup() {
  static SmallSetup s;
  return s;
}

int tile_index(int bs, int qpt) { return (bs == 256 ? 3 : 0) + (qpt == 1 ? 0 : (qpt == 2 ? 1 : 2)); }

int small_max_cluster(SmallKernel k, int bs, int qpt) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 8) {
    cudaGetLastError();
    return 0;
  }
  SmallSetup& S = small_setup();
  std::lock_guard<std::mutex> lock(S.mu);
  int& v = S.max_cluster[dev][tile_index(bs, qpt)];
  if (v >= 0) return v;
  v = 0;
  const size_t smem = small_smem_bytes(FGA_SMALL_LOOP_MAX_N, bs, qpt);
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return v;
  }
  for (int cl : {SL_MAX_CTAS, 8}) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(cl);
    cfg.blockDim = dim3(SL_NT);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) == cudaSuccess && n >= 1) {
      v = cl;
      break;
    }
    cudaGetLastError();
  }
  return v;
}

}  // namespace

bool small_loop_eligible(int64_t N, int64_t M, const DirectPlan& plan) {
  return N <= FGA_SMALL_LOOP_MAX_N && M <= FGA_SMALL_LOOP_MAX_M &&
         (double)N * (double)M <= (double)FGA_SMALL_LOOP_MAX_TERMS && small_kernel(plan.bs, plan.qpt) != nullptr &&
         plan.S >= 1 && plan.S <= 64;
}

bool small_loop_available(const DirectPlan& plan) {
  const SmallKernel k = small_kernel(plan.bs, plan.qpt);
  return k && small_max_cluster(k, plan.bs, plan.qpt) > 0;
}

int launch_small_loop(const float4* X4, int64_t N, const float4* Y0, int64_t M, DevState* ds, float eps,
                      const DirectPlan& plan, const ForceBuffers& fb, float4* V, double* partials,
                      double* traj, int traj_iters, const EpiParams& ep, unsigned long long inter_add,
                      int n_iter, cudaStream_t s) {
  if (n_iter <= 0) return FGA_OK;
  const SmallKernel k = small_kernel(plan.bs, plan.qpt);
  if (!k || !small_loop_eligible(N, M, plan)) {
    set_error("launch_small_loop: pair not eligible");
    return FGA_EINTERNAL;
  }
  const int max_cl = small_max_cluster(k, plan.bs, plan.qpt);
  if (max_cl <= 0) {
    set_error("launch_small_loop: no cluster of this kernel fits the device");
    return FGA_EINTERNAL;
  }
  const int64_t qblocks = (M + (int64_t)plan.bs * plan.qpt - 1) / ((int64_t)plan.bs * plan.qpt);
  const int64_t items = qblocks * plan.S;
  const int sub = SL_NT / plan.bs;
  const int nblk = epilogue_blocks(M);
  const int64_t want = std::max<int64_t>({(items + sub - 1) / sub, (int64_t)nblk, 1});
  const int cl = (int)std::min<int64_t>(want, max_cl);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(cl);
  cfg.blockDim = dim3(SL_NT);
  cfg.dynamicSmemBytes = small_smem_bytes(N, plan.bs, plan.qpt);
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  FGA_CUDA_TRY(cudaLaunchKernelEx(&cfg, k, X4, N, (int64_t)plan.chunk, plan.S, Y0, M, ds, eps * eps, fb.hi,
                                  fb.lo, V, partials, nblk, traj, traj_iters, ep, inter_add, n_iter));
  FGA_LAUNCH_CHECK("small_loop");
  return FGA_OK;
}

}  // namespace fga
