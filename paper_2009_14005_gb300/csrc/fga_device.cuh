// Device code of the force kernels, shared by the single-pair kernels
// (fga_force.cu) and the batched kernels (fga_batch.cu): compensated sums,
// packed FP32 pairs, template placement, the all-pairs term and the
// Barnes-Hut walks of one task. The epilogue's code (ODE step, reductions,
// rigid fit) is in fga_epi.cuh.
#pragma once

#include "fga_internal.cuh"

namespace fga {

static constexpr unsigned FULL = 0xffffffffu;

// The state before the first iteration: T = [I | 0], centroid mu0 of the
// initial template (or 0), nothing counted; finished at once if `done`.
__device__ __forceinline__ void state_init(DevState* ds, const double* __restrict__ mu0, int done) {
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
  z.done = done;
  z.converged = 0;
  z.status = 0;
  z.degenerate = 0;
  z.bh_next = 0u;
  z.bh_exited = 0u;
  *ds = z;
}

// 1/sqrt(x) from the SFU (PTX rsqrt.approx.ftz.f32). Every argument on the
// force path is r^2 + eps^2 >= eps^2 > 0, a normal number, where flushing
// subnormals changes nothing; the non-flushing form costs extra instructions
// that guard subnormal inputs.
__device__ __forceinline__ float rsqrt_fast(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Two FP32 values in one 64-bit register, and the packed FP32 instructions of
// sm_100 and later (PTX add/mul/fma .rn.f32x2): each element is computed and
// rounded exactly as the scalar instruction would, two per issue slot.
struct f2 {
  unsigned long long v;
};
__device__ __forceinline__ f2 f2_pack(float a, float b) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2_unpack(f2 r, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r.v));
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
  f2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
  return d;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
  f2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d.v) : "l"(a.v), "l"(b.v));
  return d;
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
  f2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return d;
}
__device__ __forceinline__ f2 f2_from(float4 v, int hi) {  // (x, y) or (z, w) of a float4
  return hi ? f2_pack(v.z, v.w) : f2_pack(v.x, v.y);
}

// Eq. 6 for two template points a, b (packed coordinates nya = -y) and one
// source s given as sxy = (s.x, s.x, s.y, s.y), szm = (s.z, s.z, s.m, s.m):
// adds m / (r^2 + eps^2)^(3/2) * (s - y) to (px, py, pz) of both points, with
// the same operations in the same order as the scalar loop (s.x - y.x is
// s.x + (-y.x), exactly).
__device__ __forceinline__ void pair_term2(float4 sxy, float4 szm, f2 nyx, f2 nyy, f2 nyz, f2 eps2,
                                           f2& px, f2& py, f2& pz) {
  const f2 dx = f2_add(f2_from(sxy, 0), nyx);
  const f2 dy = f2_add(f2_from(sxy, 1), nyy);
  const f2 dz = f2_add(f2_from(szm, 0), nyz);
  const f2 r2 = f2_fma(dx, dx, f2_fma(dy, dy, f2_fma(dz, dz, eps2)));
  float ra, rb;
  f2_unpack(r2, ra, rb);
  const f2 inv = f2_pack(rsqrt_fast(ra), rsqrt_fast(rb));
  const f2 w = f2_mul(f2_from(szm, 1), f2_mul(f2_mul(inv, inv), inv));
  px = f2_fma(w, dx, px);
  py = f2_fma(w, dy, py);
  pz = f2_fma(w, dz, pz);
}

// Knuth's TwoSum: s + e == a + b exactly.
__device__ __forceinline__ void comp_add(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bb = s - hi;
  const float e = (hi - (s - bb)) + (x - bb);
  hi = s;
  lo += e;
}

// x * scale rounded to the nearest integer: a value on the grid of the
// Barnes-Hut fixed-point sums (scale = 2^F, so the product is exact).
__device__ __forceinline__ long long fixed_point(float x, float scale) { return __float2ll_rn(x * scale); }

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

// ------------------------------------------------------------------ BHForce walks of one task
// Saved sibling ranges of the cooperative walk. A walk saves at most one
// range per tree level it descends below the frontier cell, and the tree has
// at most 21 levels (depth 0..20: 20-bit keys per axis, max_depth <= 20), so
// at most 20 ranges are ever saved.
constexpr int BH_DEPTH = 24;
static_assert(BH_DEPTH > 20, "the BH walk must hold one saved range per tree level");

// Per-lane BHForce of Algorithm 2 for template point y, restricted to
// frontier cell f, over the depth-first (pre-order) records: the cell's
// ancestors first (a lane accepting one stops; the monopole is added only
// when f owns the ancestor's first frontier cell), then the records
// [front[f].node, front[f].end) of f's subtree. Pre-order needs no stack: a
// record whose cell the point accepts adds its monopole and the walk skips
// its subtree (the next record is `size` further on); a rejected cell's
// first child is the next record. Single-particle records carry l^2 = -1 and
// are always accepted; a leaf holding several particles is followed by one
// record per particle, so rejecting it adds each particle exactly. Terms are
// added in the depth-first order of the per-point walk.
// Adds into the compensated accumulators (hx, lx), ... and the term count;
// `steps` is the warp's longest walk (the task's cost). A lane with
// valid == false adds nothing.
__device__ __forceinline__ void bh_task_pre(const float4* __restrict__ pcm, const float2* __restrict__ pls,
                                            const FrontCell* __restrict__ front,
                                            unsigned f, float3 y, bool valid, float eps2, float theta2,
                                            float& hx, float& hy, float& hz, float& lx, float& ly,
                                            float& lz, unsigned& count, unsigned& steps) {
  float px = 0.f, py = 0.f, pz = 0.f;
  bool live = valid;
  {
    const int npath = front[f].npath;
    const unsigned first_mask = front[f].first_mask;
    for (int j = 0; j < npath; ++j) {
      const int a = front[f].path[j];
      const float4 cm = pcm[a];
      const float l2 = pls[a].x;
      const float dx = cm.x - y.x, dy = cm.y - y.y, dz = cm.z - y.z;
      const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      const bool accept = live && l2 < theta2 * d2;
      if ((first_mask >> j) & 1u) {
        const float inv = rsqrt_fast(d2 + eps2);
        const float wgt = accept ? cm.w * (inv * inv * inv) : 0.f;
        px = fmaf(wgt, dx, px);
        py = fmaf(wgt, dy, py);
        pz = fmaf(wgt, dz, pz);
        count += accept;
      }
      live = live && !accept;
    }
  }
  const int end = front[f].end;
  int v = live ? front[f].node : end;
  unsigned n = 0;
  while (v < end) {
    const float4 cm = pcm[v];
    const float2 ri = pls[v];
    const float dx = cm.x - y.x, dy = cm.y - y.y, dz = cm.z - y.z;
    const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const bool accept = ri.x < theta2 * d2;
    const float inv = rsqrt_fast(d2 + eps2);
    const float wgt = accept ? cm.w * (inv * inv * inv) : 0.f;
    px = fmaf(wgt, dx, px);
    py = fmaf(wgt, dy, py);
    pz = fmaf(wgt, dz, pz);
    count += accept;
    v += accept ? __float_as_int(ri.y) : 1;
    if ((++n & 31u) == 0u) {
      comp_add(hx, lx, px);
      comp_add(hy, ly, py);
      comp_add(hz, lz, pz);
      px = py = pz = 0.f;
    }
  }
  comp_add(hx, lx, px);
  comp_add(hy, ly, py);
  comp_add(hz, lz, pz);
  steps += __reduce_max_sync(FULL, n);
}

// The saved ranges of the cooperative walk are spread over the warp's lanes
// (lane k holds entry k); at most 20 are ever saved (see BH_DEPTH).
static_assert(BH_DEPTH <= 32, "one saved range per lane");

// The per-point BHForce of Algorithm 2 for the 32 * NP template points of a
// warp (NP per lane), restricted to frontier cell f, walked once for the
// whole warp. Every point still takes exactly its own terms: a node is judged
// by the points that rejected all of its ancestors (bit masks m[q] over the
// lanes, one per point slot q); a point accepting the node adds its monopole,
// and the node's children are visited when at least one point rejected it,
// with the masks of the points that did. Nodes are visited depth first in
// child order, so each point adds its terms in the order of its own walk.
// The control flow is the same in every lane: a node's record is one
// broadcast load, and its bookkeeping (range, masks, saved ranges) is paid
// once for the warp's points instead of once per point.
// Adds into the compensated accumulators h[q], l[q] of point slot q and the
// term counts cnt[q]; `steps` gains the number of nodes visited (the task's
// cost).
template <int NP>
__device__ __forceinline__ void bh_walk(const float4* __restrict__ pcm, const float2* __restrict__ pls,
                                        const int2* __restrict__ pcf, const FrontCell* __restrict__ front,
                                        unsigned f, const float3 (&y)[NP], const bool (&valid)[NP], float eps2,
                                        float theta2, float (&h)[NP][3], float (&l)[NP][3],
                                        unsigned (&cnt)[NP], unsigned& steps) {
  const int lane = threadIdx.x & 31;
  const unsigned bit = 1u << lane;
  float p[NP][3];
  bool live[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    p[q][0] = p[q][1] = p[q][2] = 0.f;
    live[q] = valid[q];
  }
  {
    const int npath = front[f].npath;
    const unsigned first_mask = front[f].first_mask;
    for (int j = 0; j < npath; ++j) {
      const int a = front[f].path[j];
      const float4 cm = pcm[a];
      const float l2 = pls[a].x;
      const bool own = (first_mask >> j) & 1u;
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        const float dx = cm.x - y[q].x, dy = cm.y - y[q].y, dz = cm.z - y[q].z;
        const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const bool accept = live[q] && l2 < theta2 * d2;
        if (own) {
          const float inv = rsqrt_fast(d2 + eps2);
          const float wgt = accept ? cm.w * (inv * inv * inv) : 0.f;
          p[q][0] = fmaf(wgt, dx, p[q][0]);
          p[q][1] = fmaf(wgt, dy, p[q][1]);
          p[q][2] = fmaf(wgt, dz, p[q][2]);
          cnt[q] += accept;
        }
        live[q] = live[q] && !accept;
      }
    }
  }
  unsigned m[NP], sm[NP], any = 0u;
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    m[q] = __ballot_sync(FULL, live[q]);
    sm[q] = 0u;
    any |= m[q];
  }
  // current sibling range e = next record << 4 | cells left (siblings are a
  // subtree size apart); saved ranges and their masks: entry k in lane k's se, sm[]
  unsigned e = any != 0u ? (((unsigned)front[f].node << 4) | 1u) : 0u;
  unsigned se = 0u;
  int sp = 0;
  // NP == 2: packed coordinates -y of the two points, and packed partial sums
  // (which take over the ancestors' terms; p is unpacked from them before
  // every use)
  const f2 nyx = f2_pack(-y[0].x, -y[NP - 1].x), nyy = f2_pack(-y[0].y, -y[NP - 1].y);
  const f2 nyz = f2_pack(-y[0].z, -y[NP - 1].z);
  const f2 th2 = f2_pack(theta2, theta2), e2 = f2_pack(eps2, eps2);
  f2 px2 = f2_pack(p[0][0], p[NP - 1][0]), py2 = f2_pack(p[0][1], p[NP - 1][1]);
  f2 pz2 = f2_pack(p[0][2], p[NP - 1][2]);
  while ((e & 15u) != 0u) {
    ++steps;
    const int v = (int)(e >> 4);
    const float4 cm = pcm[v];
    const float2 ri = pls[v];
    const int nchild = pcf[v].x;
    e += ((unsigned)__float_as_int(ri.y) << 4) - 1u;  // next sibling
    bool rej[NP];
    unsigned r[NP], rany = 0u;
    if constexpr (NP == 2) {
      // both points judge the same cell: the packed FP32 instructions take
      // them together, each element as the scalar code below computes it
      const f2 dx = f2_add(f2_pack(cm.x, cm.x), nyx), dy = f2_add(f2_pack(cm.y, cm.y), nyy);
      const f2 dz = f2_add(f2_pack(cm.z, cm.z), nyz);
      const f2 d2 = f2_fma(dx, dx, f2_fma(dy, dy, f2_mul(dz, dz)));
      const f2 od2 = f2_mul(th2, d2);
      float o0, o1, e0, e1;
      f2_unpack(od2, o0, o1);
      f2_unpack(f2_add(d2, e2), e0, e1);
      const bool act0 = (m[0] & bit) != 0u, act1 = (m[1] & bit) != 0u;
      const bool acc0 = act0 && ri.x < o0, acc1 = act1 && ri.x < o1;
      const f2 inv = f2_pack(rsqrt_fast(e0), rsqrt_fast(e1));
      const f2 w = f2_mul(f2_pack(cm.w, cm.w), f2_mul(f2_mul(inv, inv), inv));
      float w0, w1;
      f2_unpack(w, w0, w1);
      const f2 wsel = f2_pack(acc0 ? w0 : 0.f, acc1 ? w1 : 0.f);
      px2 = f2_fma(wsel, dx, px2);
      py2 = f2_fma(wsel, dy, py2);
      pz2 = f2_fma(wsel, dz, pz2);
      cnt[0] += acc0;
      cnt[1] += acc1;
      rej[0] = act0 && !acc0;
      rej[1] = act1 && !acc1;
      r[0] = __ballot_sync(FULL, rej[0]);
      r[1] = __ballot_sync(FULL, rej[1]);
      rany = r[0] | r[1];
    } else {
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        const bool act = (m[q] & bit) != 0u;
        const float dx = cm.x - y[q].x, dy = cm.y - y[q].y, dz = cm.z - y[q].z;
        const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        // single-particle records carry l^2 = -1: always accepted (one exact term)
        const bool accept = act && ri.x < theta2 * d2;
        const float inv = rsqrt_fast(d2 + eps2);
        const float wgt = accept ? cm.w * (inv * inv * inv) : 0.f;
        p[q][0] = fmaf(wgt, dx, p[q][0]);
        p[q][1] = fmaf(wgt, dy, p[q][1]);
        p[q][2] = fmaf(wgt, dz, p[q][2]);
        cnt[q] += accept;
        rej[q] = act && !accept;
        r[q] = __ballot_sync(FULL, rej[q]);
        rany |= r[q];
      }
    }
    if (rany != 0u) {
      if (nchild > 0) {
        // descend: save the rest of the current range, continue with the
        // children (the first follows its parent), judged by the points that
        // rejected this cell
        if ((e & 15u) != 0u) {
          if (lane == sp) {
            se = e;
#pragma unroll
            for (int q = 0; q < NP; ++q) sm[q] = m[q];
          }
          ++sp;
        }
        e = ((unsigned)(v + 1) << 4) | (unsigned)nchild;
#pragma unroll
        for (int q = 0; q < NP; ++q) m[q] = r[q];
      } else if (nchild < -1) {
        // leaf holding several particles, rejected by these points: each
        // particle exactly, from the single-particle records that follow it (rare)
        const int nb = -nchild;
        if constexpr (NP == 2) {
          f2_unpack(px2, p[0][0], p[1][0]);
          f2_unpack(py2, p[0][1], p[1][1]);
          f2_unpack(pz2, p[0][2], p[1][2]);
        }
        for (int b = 1; b <= nb; ++b) {
          const float4 qb = pcm[v + b];
#pragma unroll
          for (int q = 0; q < NP; ++q) {
            const float ex = qb.x - y[q].x, ey = qb.y - y[q].y, ez = qb.z - y[q].z;
            const float iq = rsqrt_fast(fmaf(ex, ex, fmaf(ey, ey, fmaf(ez, ez, eps2))));
            const float wq = rej[q] ? qb.w * (iq * iq * iq) : 0.f;
            p[q][0] = fmaf(wq, ex, p[q][0]);
            p[q][1] = fmaf(wq, ey, p[q][1]);
            p[q][2] = fmaf(wq, ez, p[q][2]);
          }
        }
#pragma unroll
        for (int q = 0; q < NP; ++q) cnt[q] += rej[q] ? (unsigned)nb : 0u;
        if constexpr (NP == 2) {
          px2 = f2_pack(p[0][0], p[1][0]);
          py2 = f2_pack(p[0][1], p[1][1]);
          pz2 = f2_pack(p[0][2], p[1][2]);
        }
      }
    }
    // range exhausted: resume the innermost saved range
    if ((e & 15u) == 0u && sp > 0) {
      --sp;
      e = __shfl_sync(FULL, se, sp);
#pragma unroll
      for (int q = 0; q < NP; ++q) m[q] = __shfl_sync(FULL, sm[q], sp);
    }
    if ((steps & 31u) == 0u) {
      if constexpr (NP == 2) {
        f2_unpack(px2, p[0][0], p[1][0]);
        f2_unpack(py2, p[0][1], p[1][1]);
        f2_unpack(pz2, p[0][2], p[1][2]);
        px2 = py2 = pz2 = f2_pack(0.f, 0.f);
      }
#pragma unroll
      for (int q = 0; q < NP; ++q)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          comp_add(h[q][c], l[q][c], p[q][c]);
          p[q][c] = 0.f;
        }
    }
  }
  if constexpr (NP == 2) {
    f2_unpack(px2, p[0][0], p[1][0]);
    f2_unpack(py2, p[0][1], p[1][1]);
    f2_unpack(pz2, p[0][2], p[1][2]);
  }
#pragma unroll
  for (int q = 0; q < NP; ++q)
#pragma unroll
    for (int c = 0; c < 3; ++c) comp_add(h[q][c], l[q][c], p[q][c]);
}

// The per-point BHForce of Algorithm 2 for the 32 * NP template points of a
// warp (NP = 1, 2 or 4 per lane), restricted to frontier cell f, as one walk
// that follows all the points' own walks at once. Each point keeps the
// position of its own stackless depth-first walk (bh_task_pre): the record
// it reads next, nx. The warp reads the smallest nx over its points (one
// broadcast record load); the points whose walk is at that record judge it
// exactly as their own walk would (accept: add the monopole, skip the
// subtree; reject: go to the next record), the others wait. Since every walk
// only moves forward through the pre-order records, the warp visits exactly
// the union of its points' walks, in order, and each point adds exactly its
// own terms in its own order. (A point waiting beyond record v accepted an
// ancestor of v, so the next record is always v + 1 if some point rejected v
// and v + size(v) otherwise; with FGA_BH_CURSOR_VOTE the warp takes it from a
// vote instead of the minimum.) Per step: one record, one judgement per point
// (packed FP32 pairs for NP >= 2) and one warp-wide reduction; no stack, no
// masks.
// Partial sums are flushed into the compensated accumulators every 32 warp
// steps. Adds into h[q], l[q], cnt[q]; `steps` gains the records visited.
#ifndef FGA_BH_CURSOR_VOTE
#define FGA_BH_CURSOR_VOTE 0
#endif

template <int NP>
__device__ __forceinline__ void bh_walk_cursor(const float4* __restrict__ pcm,
                                               const float2* __restrict__ pls,
                                               const FrontCell* __restrict__ front, unsigned f,
                                               const float3 (&y)[NP], const bool (&valid)[NP],
                                               float eps2, float theta2, float (&h)[NP][3],
                                               float (&l)[NP][3], unsigned (&cnt)[NP],
                                               unsigned& steps) {
  static_assert(NP == 1 || NP == 2 || NP == 4, "one, two or four points per lane");
  float p[NP][3];
  bool live[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    p[q][0] = p[q][1] = p[q][2] = 0.f;
    live[q] = valid[q];
  }
  {
    const int npath = front[f].npath;
    const unsigned first_mask = front[f].first_mask;
    for (int j = 0; j < npath; ++j) {
      const int a = front[f].path[j];
      const float4 cm = pcm[a];
      const float l2 = pls[a].x;
      const bool own = (first_mask >> j) & 1u;
#pragma unroll
      for (int q = 0; q < NP; ++q) {
        const float dx = cm.x - y[q].x, dy = cm.y - y[q].y, dz = cm.z - y[q].z;
        const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const bool accept = live[q] && l2 < theta2 * d2;
        if (own) {
          const float inv = rsqrt_fast(d2 + eps2);
          const float wgt = accept ? cm.w * (inv * inv * inv) : 0.f;
          p[q][0] = fmaf(wgt, dx, p[q][0]);
          p[q][1] = fmaf(wgt, dy, p[q][1]);
          p[q][2] = fmaf(wgt, dz, p[q][2]);
          cnt[q] += accept;
        }
        live[q] = live[q] && !accept;
      }
    }
  }
  const int end = front[f].end;
  int nx[NP];
  int first = end;
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    nx[q] = live[q] ? front[f].node : end;
    first = min(first, nx[q]);
  }
  int v = (int)__reduce_min_sync(FULL, (unsigned)first);
  unsigned k = 0;
  if constexpr (NP >= 2) {
    constexpr int NR = NP / 2;  // packed pairs of points (2r, 2r + 1)
    f2 nyx[NR], nyy[NR], nyz[NR], px2[NR], py2[NR], pz2[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      nyx[r] = f2_pack(-y[2 * r].x, -y[2 * r + 1].x);
      nyy[r] = f2_pack(-y[2 * r].y, -y[2 * r + 1].y);
      nyz[r] = f2_pack(-y[2 * r].z, -y[2 * r + 1].z);
      px2[r] = f2_pack(p[2 * r][0], p[2 * r + 1][0]);
      py2[r] = f2_pack(p[2 * r][1], p[2 * r + 1][1]);
      pz2[r] = f2_pack(p[2 * r][2], p[2 * r + 1][2]);
    }
    const f2 th2 = f2_pack(theta2, theta2), e2 = f2_pack(eps2, eps2);
    // one record of the union walk: every point at record v judges it
    auto step = [&]() {
      const float4 cm = pcm[v];
      const float2 ri = pls[v];
      const int skip = __float_as_int(ri.y);
      const f2 cx = f2_pack(cm.x, cm.x), cy = f2_pack(cm.y, cm.y), cz = f2_pack(cm.z, cm.z);
      const f2 cw = f2_pack(cm.w, cm.w);
      const int v_acc = v + skip, v_rej = v + 1;
      int lo = end;
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const f2 dx = f2_add(cx, nyx[r]), dy = f2_add(cy, nyy[r]), dz = f2_add(cz, nyz[r]);
        const f2 d2 = f2_fma(dx, dx, f2_fma(dy, dy, f2_mul(dz, dz)));
        float o0, o1, e0, e1;
        f2_unpack(f2_mul(th2, d2), o0, o1);
        f2_unpack(f2_add(d2, e2), e0, e1);
        const bool act0 = nx[2 * r] == v, act1 = nx[2 * r + 1] == v;
        const bool acc0 = act0 && ri.x < o0, acc1 = act1 && ri.x < o1;
        const f2 inv = f2_pack(rsqrt_fast(e0), rsqrt_fast(e1));
        const f2 w = f2_mul(cw, f2_mul(f2_mul(inv, inv), inv));
        float w0, w1;
        f2_unpack(w, w0, w1);
        const f2 wsel = f2_pack(acc0 ? w0 : 0.f, acc1 ? w1 : 0.f);
        px2[r] = f2_fma(wsel, dx, px2[r]);
        py2[r] = f2_fma(wsel, dy, py2[r]);
        pz2[r] = f2_fma(wsel, dz, pz2[r]);
        cnt[2 * r] += acc0;
        cnt[2 * r + 1] += acc1;
        nx[2 * r] = act0 ? (acc0 ? v_acc : v_rej) : nx[2 * r];
        nx[2 * r + 1] = act1 ? (acc1 ? v_acc : v_rej) : nx[2 * r + 1];
        lo = min(lo, min(nx[2 * r], nx[2 * r + 1]));
      }
#if FGA_BH_CURSOR_VOTE
      {
        bool rej = false;
#pragma unroll
        for (int q = 0; q < NP; ++q) rej = rej || nx[q] == v_rej;
        v = __any_sync(FULL, rej) ? v_rej : v_acc;
      }
#else
      v = (int)__reduce_min_sync(FULL, (unsigned)lo);
#endif
    };
    // four records per pass (v is the same in every lane, so the exits are
    // uniform), the FP32 sums flushed every 32 records
    while (v < end) {
      step();
      ++k;
      if (v >= end) break;
      step();
      ++k;
      if (v >= end) break;
      step();
      ++k;
      if (v >= end) break;
      step();
      ++k;
      if ((k & 31u) == 0u) {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          f2_unpack(px2[r], p[2 * r][0], p[2 * r + 1][0]);
          f2_unpack(py2[r], p[2 * r][1], p[2 * r + 1][1]);
          f2_unpack(pz2[r], p[2 * r][2], p[2 * r + 1][2]);
          px2[r] = py2[r] = pz2[r] = f2_pack(0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < NP; ++q)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            comp_add(h[q][c], l[q][c], p[q][c]);
            p[q][c] = 0.f;
          }
      }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      f2_unpack(px2[r], p[2 * r][0], p[2 * r + 1][0]);
      f2_unpack(py2[r], p[2 * r][1], p[2 * r + 1][1]);
      f2_unpack(pz2[r], p[2 * r][2], p[2 * r + 1][2]);
    }
  } else {
    while (v < end) {
      const float4 cm = pcm[v];
      const float2 ri = pls[v];
      const int skip = __float_as_int(ri.y);
      const float dx = cm.x - y[0].x, dy = cm.y - y[0].y, dz = cm.z - y[0].z;
      const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      const bool act = nx[0] == v;
      const bool accept = act && ri.x < theta2 * d2;
      const float inv = rsqrt_fast(d2 + eps2);
      const float wgt = accept ? cm.w * (inv * inv * inv) : 0.f;
      p[0][0] = fmaf(wgt, dx, p[0][0]);
      p[0][1] = fmaf(wgt, dy, p[0][1]);
      p[0][2] = fmaf(wgt, dz, p[0][2]);
      cnt[0] += accept;
      nx[0] = act ? v + (accept ? skip : 1) : nx[0];
#if FGA_BH_CURSOR_VOTE
      v = __any_sync(FULL, act && !accept) ? v + 1 : v + skip;
#else
      v = (int)__reduce_min_sync(FULL, (unsigned)nx[0]);
#endif
      if ((++k & 31u) == 0u) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          comp_add(h[0][c], l[0][c], p[0][c]);
          p[0][c] = 0.f;
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < NP; ++q)
#pragma unroll
    for (int c = 0; c < 3; ++c) comp_add(h[q][c], l[q][c], p[q][c]);
  steps += k;
}

}  // namespace fga
