// fga_forces_direct_static: the all-pairs force of fga_forces for callers that
// cannot allocate device memory.
//
// Who needs it: a caller that must never enter the device allocator. Examples
// are a control loop with a hard latency budget (cudaMalloc / cudaFree can
// block and synchronise the device), and a plug-in inside a host application
// that has already handed all device memory to its own pool. Such callers
// still pass their own inputs and outputs; only the intermediate buffers move
// into one fixed array compiled into this library.
//
// The array is a file-scope __device__ array, so every GPU that loads the
// library holds it (8 MiB) until the process exits. Host code cannot pass the
// array's name to a kernel (on the host that name is only a stand-in, not a
// device address), so every call looks up the array's device address on the
// current device with cudaGetSymbolAddress, a host-side query that allocates
// nothing. Looking it up on every call (rather than caching it per device)
// keeps the address right when the module is loaded again, after a
// cudaDeviceReset or under another context. The first call on a device loads
// the library's device code there; make it before any stream capture.
#include <algorithm>
#include <string>

#include "fga_internal.cuh"

namespace fga {

static __device__ __align__(256) float4 g_static_scratch[FGA_STATIC_SCRATCH_FLOAT4];

// Device address of g_static_scratch on the current device.
static int static_scratch(float4** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    set_error(std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
    return FGA_ECUDA;
  }
  *out = static_cast<float4*>(p);
  return FGA_OK;
}

__global__ void k_static_pack(const float* __restrict__ xyz, const float* __restrict__ m,
                              float m_default, int64_t n, float4* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = make_float4(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], m ? m[i] : m_default);
}

// float4 slots taken by one DevState at the start of the array
static constexpr int64_t kStateSlots = (int64_t)((sizeof(DevState) + sizeof(float4) - 1) / sizeof(float4));
static_assert(kStateSlots == FGA_STATIC_STATE_FLOAT4, "the header's state-block size is out of date");

static int64_t footprint(int64_t N, int64_t M, int S) { return kStateSlots + N + M + 2 * (int64_t)S * M; }

}  // namespace fga

using namespace fga;

extern "C" int fga_forces_direct_static(const float* X, const float* mX, int64_t N, const float* Y,
                                        const float* mY, int64_t M, const fga_params* p,
                                        float* acc_out, void* stream) {
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  if (!p || !(p->eps > 0.f) || N <= 0 || M <= 0 || !X || !Y || !acc_out) {
    set_error("fga_forces_direct_static: bad arguments");
    return FGA_EINVAL;
  }
  // same split plan as fga_forces; one source split if that does not fit
  DirectPlan plan = plan_direct(N, M);
  if (footprint(N, M, plan.S) > FGA_STATIC_SCRATCH_FLOAT4) {
    plan.S = 1;
    plan.chunk = (N + plan.bs - 1) / plan.bs * plan.bs;
  }
  if (footprint(N, M, plan.S) > FGA_STATIC_SCRATCH_FLOAT4) {
    set_error("fga_forces_direct_static: N + M + 2*M + " + std::to_string(kStateSlots) +
              " float4 exceed the static scratch of " + std::to_string(FGA_STATIC_SCRATCH_FLOAT4) +
              " float4 (N = " + std::to_string(N) + ", M = " + std::to_string(M) + ")");
    return FGA_EINVAL;
  }
  float4* base = nullptr;
  int rc = static_scratch(&base);
  if (rc) return rc;
  DevState* ds = reinterpret_cast<DevState*>(base);
  float4* X4 = base + kStateSlots;
  float4* Y0 = X4 + N;
  ForceBuffers fb;
  fb.hi = Y0 + M;
  fb.lo = fb.hi + (int64_t)plan.S * M;
  fb.S = plan.S;
  const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, 8 * (int64_t)sm_count()));
  const unsigned gy = (unsigned)std::max<int64_t>(1, std::min<int64_t>((M + 255) / 256, 8 * (int64_t)sm_count()));
  // Every region read below is rewritten first: the state block by
  // launch_state_init (identity transform, flags cleared), the packed inputs
  // by k_static_pack, and each partial sum by the force kernel.
  k_static_pack<<<gx, 256, 0, s>>>(X, mX, (float)(1.0 / (double)N), N, X4);
  FGA_LAUNCH_CHECK("static_pack X");
  k_static_pack<<<gy, 256, 0, s>>>(Y, mY, 1.0f, M, Y0);
  FGA_LAUNCH_CHECK("static_pack Y");
  if ((rc = launch_state_init(ds, nullptr, s))) return rc;
  if ((rc = launch_direct(X4, N, Y0, M, ds, p->eps, plan, fb, s))) return rc;
  return launch_forces_out(fb, M, Y0, mY != nullptr, p->G, nullptr, acc_out, s);
}
