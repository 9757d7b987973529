// Device code shared by the single-pair kernels (fga_force.cu) and the
// batched kernels (fga_batch.cu): compensated sums, template placement, the
// per-task Barnes-Hut walk, the per-point ODE step with its reduction terms,
// and the FP64 rigid fit of one iteration.
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

// Symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations (FP64):
// A = V diag(w) V^T, eigenvalues sorted descending, eigenvectors in V's columns.
static __device__ void eig_sym3(const double A_in[9], double w[3], double V[9]) {
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
static __device__ bool rigid_rotation(const double C[9], double R[9]) {
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
static __device__ bool polar_rotation(const double C[9], double R[9]) {
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

// Eq. 14 for D = 2 (clouds in a plane z = const): the rotation R' of the
// plane maximising tr(R'^T C2) over the x, y block C2 of C, i.e. the angle
// atan2(c21 - c12, c11 + c22), embedded as diag(R', 1). False (no unique
// optimum: every rotation fits equally) when both arguments vanish.
__device__ __forceinline__ bool planar_rotation(const double C[9], double R[9]) {
  const double c11 = C[0], c12 = C[1], c21 = C[3], c22 = C[4];
  const double p = c11 + c22, q = c21 - c12;
  const double r = sqrt(p * p + q * q);
  const double fro = sqrt(c11 * c11 + c12 * c12 + c21 * c21 + c22 * c22);
  if (!(r > 1e-12 * fro)) return false;
  const double c = p / r, s = q / r;
  R[0] = c;
  R[1] = -s;
  R[2] = 0.0;
  R[3] = s;
  R[4] = c;
  R[5] = 0.0;
  R[6] = 0.0;
  R[7] = 0.0;
  R[8] = 1.0;
  return true;
}

// One thread: reductions -> C -> (R', t') -> compose, convergence, next-iteration constants.
static __device__ void rigid_step(const double* red, int64_t M, DevState* ds, const EpiParams& ep,
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
  const bool ok = ep.dim == 2 ? planar_rotation(C, Rp) : (polar_rotation(C, Rp) || rigid_rotation(C, Rp));
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
    if (ep.conv_tol > 0 && d2 <= ep.conv_tol) {
      ds->done = 1;
      ds->converged = 1;
    }
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
  if (ep.max_iter > 0 && k_it + 1 >= ep.max_iter) ds->done = 1;
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
__device__ __forceinline__ void bh_task_pre(const float4* __restrict__ pre, const FrontCell* __restrict__ front,
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
      const float4 cm = pre[2 * a];
      const float l2 = pre[2 * a + 1].x;
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
    const float4 cm = pre[2 * v];
    const float4 ri = pre[2 * v + 1];
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
__device__ __forceinline__ void bh_walk(const float4* __restrict__ pre, const FrontCell* __restrict__ front,
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
      const float4 cm = pre[2 * a];
      const float l2 = pre[2 * a + 1].x;
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
    const float4 cm = pre[2 * v];
    const float4 ri = pre[2 * v + 1];
    const int nchild = __float_as_int(ri.z);
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
          const float4 qb = pre[2 * (v + b)];
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

// ------------------------------------------------------------------ epilogue stages
constexpr int EPI_BS = 256;  // threads per epilogue block

struct EpiCtx {
  Xf xf;
  float mu[3];      // FP32 centre subtracted from the template points
  float A[9], b[3]; // rigid-velocity coefficients (velocity_mode RIGID)
};

__device__ __forceinline__ EpiCtx load_epi(const DevState* __restrict__ ds) {
  EpiCtx c;
  c.xf = load_xf(ds);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    c.mu[k] = ds->muf[k];
    c.b[k] = ds->b[k];
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) c.A[k] = ds->A[k];
  return c;
}

// Template point i: a = G * (compensated sum of the S force partials);
// Eq. 9 with the dissipative force of Eq. 7, v' = v + dt (a - eta v / m_Y);
// Eq. 10, d = dt v'. Adds the point's 27 reduction terms to r: centred
// position yc, d, yc yc^T (6), d yc^T (9), force m_Y a, torque yc x m_Y a.
// `live`: bit s set for the slots to add (all S slots when no mask is kept);
// the others are exact zeros, and adding a zero never changes a compensated
// sum, so the result is the same as adding all S slots in order.
__device__ __forceinline__ void epi_point(int64_t i, const float4* __restrict__ Y0,
                                          const float4* __restrict__ hi, const float4* __restrict__ lo,
                                          int S, int64_t M, float4* __restrict__ V,
                                          const EpiParams& ep, const EpiCtx& c, float (&r)[NRED],
                                          unsigned long long live = ~0ull) {
  const float4 y0 = Y0[i];
  const float3 y = place(c.xf, y0);
  const float cx = y.x - c.mu[0], cy = y.y - c.mu[1], cz = y.z - c.mu[2];
  float ahx = 0.f, ahy = 0.f, ahz = 0.f, alx = 0.f, aly = 0.f, alz = 0.f;
  if (S <= 64 && live != ~0ull) {
    unsigned long long rest = live & (S == 64 ? ~0ull : ((1ull << S) - 1ull));
    while (rest) {
      // up to four slots in flight, then the same in-order compensated sum
      int sl[4];
      int nk = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        sl[k] = rest ? __ffsll((long long)rest) - 1 : -1;
        if (rest) {
          rest &= rest - 1ull;
          ++nk;
        }
      }
      float4 h[4], l[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        h[k] = sl[k] >= 0 ? hi[(int64_t)sl[k] * M + i] : make_float4(0.f, 0.f, 0.f, 0.f);
        l[k] = sl[k] >= 0 ? lo[(int64_t)sl[k] * M + i] : make_float4(0.f, 0.f, 0.f, 0.f);
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
      (void)nk;
    }
  } else {
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
  }
  const float ax = ep.G * (ahx + alx), ay = ep.G * (ahy + aly), az = ep.G * (ahz + alz);
  float vx, vy, vz;
  if (ep.vmode == FGA_VEL_RIGID) {
    vx = fmaf(c.A[0], y.x, fmaf(c.A[1], y.y, fmaf(c.A[2], y.z, c.b[0])));
    vy = fmaf(c.A[3], y.x, fmaf(c.A[4], y.y, fmaf(c.A[5], y.z, c.b[1])));
    vz = fmaf(c.A[6], y.x, fmaf(c.A[7], y.y, fmaf(c.A[8], y.z, c.b[2])));
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

// Block partial of r: FP32 within each warp (a few dozen terms), FP64 across
// the block's warps in a fixed order; NRED doubles written to out. Every
// thread of the block must call it.
__device__ __forceinline__ void epi_block_partial(float (&r)[NRED], double* __restrict__ out) {
  __shared__ double s_w[EPI_BS / 32][NRED];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
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
    out[threadIdx.x] = acc;
  }
}

// FP64 sum of nblocks x NRED partials in a fixed order, by the whole block:
// thread t < 8 NRED adds value t % NRED over blocks t / NRED, + 8, ...;
// NRED threads then add the 8 strands into s_red (shared, NRED doubles).
// FP64 adds are scarce on this GPU, so no FP64 warp shuffles are used.
__device__ __forceinline__ void epi_last_reduce(const double* partials, int nblocks, double* s_red) {
  __shared__ double s_strand[8][NRED];
  if (threadIdx.x < 8 * NRED) {
    const int k = threadIdx.x % NRED, j = threadIdx.x / NRED;
    double acc = 0.0;
    for (int b = j; b < nblocks; b += 8) acc += __ldcg(&partials[(int64_t)b * NRED + k]);
    s_strand[j][k] = acc;
  }
  __syncthreads();
  if (threadIdx.x < NRED) {
    double acc = 0.0;
    for (int j = 0; j < 8; ++j) acc += s_strand[j][threadIdx.x];
    s_red[threadIdx.x] = acc;
  }
  __syncthreads();
}

}  // namespace fga
