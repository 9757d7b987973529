// Many independent pairs in one launch: the per-pair descriptor, its setup and
// the launch helpers shared by the batch executor (fga_batch.cu) and the
// serving engine (fga_serve.cu). Host-side declarations only.
#pragma once

#include <vector>

#include "fga_internal.cuh"

namespace fga {

constexpr int BATCH_CHUNK = 2048;  // reference points per all-pairs task
constexpr int BATCH_BH_GROUP = 32;  // template points per Barnes-Hut task (one per lane)
constexpr int BATCH_WARPS = 4;

// Everything the two batch kernels need about one pair, in device memory.
struct PairDev {
  int method;                 // FGA_DIRECT or FGA_BH
  int K;                      // BH: frontier cells; direct: source chunks
  const float4* pcm;          // BH: depth-first cell records (CoM, mass)
  const float2* pls;          // BH: depth-first cell records (l^2, subtree size)
  const FrontCell* front;     // BH: frontier (record indices)
  const float4* X4;           // direct: reference points and masses
  int64_t N, M;
  const float4* Y0;           // template points and masses
  DevState* ds;
  float4* hi;                 // K x M compensated partial sums
  float4* lo;
  float4* V;
  double* partials;           // nblk x NRED
  unsigned* counter;          // epilogue blocks finished
  int nblk;                   // epilogue blocks of this pair
  EpiParams ep;
  unsigned long long inter_add;  // direct: N*M terms per iteration
  float eps2, theta2;            // this pair's softening and opening parameters, squared
};

// Builds the resident data of one prepared pair (tree or packed reference,
// packed template, velocities, partial-sum buffers) into `keep`, initialises
// the state `ds` (device memory of one DevState) and fills the descriptor P.
// The tree, if any, is returned in *tree (owned by the caller).
int build_pair(const fga_pair& q, const Prepared& pr, const fga_params* p, Scratch& keep,
               fga_tree** tree, DevState* ds, PairDev& P, cudaStream_t s);
// The two halves of build_pair. build_inputs: the read-only inputs of the
// pair (method, tree or packed reference, packed template, its centroid in
// *mu0), which pairs with the same inputs may share. build_state: this pair's
// own state, velocities, partial sums and parameters, on inputs already in P.
int build_inputs(const fga_pair& q, const Prepared& pr, const fga_params* p, Scratch& keep,
                 fga_tree** tree, PairDev& P, double** mu0, cudaStream_t s);
int build_state(const fga_params* p, const double* mu0, Scratch& keep, DevState* ds, PairDev& P,
                cudaStream_t s);

// Work layout of a batch of pairs (in the order of `pairs`): pair k owns warp
// tasks task_start[k] .. task_start[k+1]-1 (task = group * K + f: a group of
// 32 template points and frontier cell f for Barnes-Hut, of 64 points and
// reference chunk f for the all-pairs sum) and epilogue blocks
// block_start[k] .. block_start[k+1]-1. Both arrays get pairs.size() + 1
// entries. Returns false if a count exceeds 2^31.
bool batch_layout(const std::vector<PairDev>& pairs, std::vector<unsigned>& task_start,
                  std::vector<unsigned>& block_start);

// Checks the eight device flags prepare_inputs wrote for pair k (host copy);
// returns FGA_OK or FGA_EINVAL with the message set.
int check_pair_flags(const int* f, const char* who, int64_t k);

// Result of one pair from its final state and normalisation record.
void fill_pair_result(const DevState& h, const double* info, int method, const fga_params* p,
                      fga_pair_result& r);

// Upper bound of the device bytes one pair holds while it is resident (and
// while it is being prepared), for memory admission.
int64_t pair_bytes_bound(int64_t N, int64_t M, int method, const fga_params* p);

// Grid of the batch force kernel for ntasks warp tasks.
int batch_force_grid(unsigned ntasks);

// One iteration of Algorithm 2 for every pair of the batch: the force launch
// over task_start[npairs] tasks, then the epilogue launch over
// block_start[npairs] blocks (device copies of batch_layout's arrays; ntasks
// and nblocks are their last entries; 0 skips that launch). d_ctr: two
// unsigned counters, zero before the first launch (the force kernel leaves
// them zero). Pairs whose state is `done` skip their work.
// order/cost: the heavy-first task order (slot -> task) or null, and where
// each task's cost is recorded, or null (see launch_task_order).
int launch_batch_iteration(const PairDev* d_pairs, int npairs, const unsigned* d_task_start,
                           unsigned ntasks, const unsigned* d_block_start, unsigned nblocks,
                           unsigned* d_ctr, int fgrid, cudaStream_t s,
                           const unsigned* order = nullptr, unsigned* cost = nullptr);


// out[k] = pairs[k].ds->done for k < n.
int launch_done_flags(const PairDev* d_pairs, int n, int* d_out, cudaStream_t s);

}  // namespace fga
