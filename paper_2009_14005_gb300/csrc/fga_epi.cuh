// Device code of the epilogue, shared by the single-pair kernels
// (fga_force.cu) and the batched kernels (fga_batch.cu): the per-point ODE
// step with its reduction terms (Eqs. 7-10), the block and cross-block FP64
// reductions, and the FP64 rigid fit of one iteration (Eqs. 14, 16) with the
// composition of the transform and the stop test.
#pragma once

#include "fga_device.cuh"

namespace fga {

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

// FP64 on this GPU: an FP64 instruction (add, multiply, FMA, and the
// conversions to and from FP32) occupies its warp's FP64 pipe for about 64
// cycles, however few of the warp's lanes are active (measured: the same 64
// cycles per instruction with 1, 9 or 32 active lanes, and for dependent or
// independent operations). So the rigid fit spreads its 3 x 3 matrices over
// the lanes of a warp, one entry per lane, and each FP64 step of it is one
// instruction for all nine entries. Reciprocals are an FP32 seed refined by
// two Newton steps in FP64 (r <- r + r (1 - d r), 24 -> 48 -> 53 bits).
__device__ __forceinline__ double rcp64(double d) {
  double r = (double)__frcp_rn((float)d);
  r = fma(r, fma(-d, r, 1.0), r);
  r = fma(r, fma(-d, r, 1.0), r);
  return r;
}

// Cofactor matrix of X (returned det X): entry (r, c) is
// X[r1][c1] X[r2][c2] - X[r1][c2] X[r2][c1] with r1, r2 = r + 1, r + 2 and
// c1, c2 = c + 1, c + 2 (mod 3).
template <class T>
__device__ __forceinline__ T cof3(const T X[9], T cf[9]) {
  cf[0] = X[4] * X[8] - X[5] * X[7];
  cf[1] = X[5] * X[6] - X[3] * X[8];
  cf[2] = X[3] * X[7] - X[4] * X[6];
  cf[3] = X[2] * X[7] - X[1] * X[8];
  cf[4] = X[0] * X[8] - X[2] * X[6];
  cf[5] = X[1] * X[6] - X[0] * X[7];
  cf[6] = X[1] * X[5] - X[2] * X[4];
  cf[7] = X[2] * X[3] - X[0] * X[5];
  cf[8] = X[0] * X[4] - X[1] * X[3];
  return X[0] * cf[0] + X[1] * cf[1] + X[2] * cf[2];  // det X
}

// Sum of entries 0..8 held one per lane (lanes 0..8), in the order
// ((v0 + v1) + (v2 + v3)) + ((v4 + v5) + (v6 + v7)) + v8; the same in every lane.
__device__ __forceinline__ double lane_sum9(double v) {
  const double a1 = v + __shfl_down_sync(FULL, v, 1);
  const double a2 = a1 + __shfl_down_sync(FULL, a1, 2);
  const double a3 = a2 + __shfl_down_sync(FULL, a2, 4);
  return __shfl_sync(FULL, a3 + __shfl_sync(FULL, v, 8), 0);
}

// Entry k of a 3 x 3 matrix held in registers by every lane.
template <class T>
__device__ __forceinline__ T pick9(const T (&A)[9], int k) {
  T v = A[0];
#pragma unroll
  for (int j = 1; j < 9; ++j) v = k == j ? A[j] : v;
  return v;
}

// Cofactor (r, c) of a 3 x 3 matrix held one entry per lane (lane 3 r + c):
// a[r1][c1] a[r2][c2] - a[r1][c2] a[r2][c1] with r1, r2 = r + 1, r + 2 and c1,
// c2 = c + 1, c + 2 (mod 3); det = a0 cf0 + a1 cf1 + a2 cf2 in every lane.
__device__ __forceinline__ double lane_cof3(double a, int r1, int r2, int c1, int c2, double& det) {
  const double xa = __shfl_sync(FULL, a, 3 * r1 + c1), xb = __shfl_sync(FULL, a, 3 * r2 + c2);
  const double xc = __shfl_sync(FULL, a, 3 * r1 + c2), xd = __shfl_sync(FULL, a, 3 * r2 + c1);
  const double cf = xa * xb - xc * xd;
  det = __shfl_sync(FULL, a, 0) * __shfl_sync(FULL, cf, 0) + __shfl_sync(FULL, a, 1) * __shfl_sync(FULL, cf, 1) +
        __shfl_sync(FULL, a, 2) * __shfl_sync(FULL, cf, 2);
  return cf;
}

// Orthogonal polar factor of C by Newton's iteration X <- (X + X^{-T}) / 2
// (Higham), started from a positive multiple of C. For det C > 0 the limit is
// U V^T of C = U S V^T, i.e. Eq. 14's rotation (sgn det(U V^T) = +1). The
// first, scaled steps X <- (g X + X^{-T} / g) / 2, g = (|X^{-1}|_F /
// |X|_F)^{1/2} (any g > 0 keeps the limit), run in FP32 until the iterate is
// within about 1e-6 of U V^T; unscaled FP64 steps then converge quadratically
// to the FP64 fixed point: from a converged FP32 iterate (error about 1e-7)
// one step leaves an orthogonal matrix to FP64 precision, so one step is
// taken (otherwise steps repeat until they stop moving); a last correction
// against C (below) then moves it onto C's own polar factor.
// Called by all 32 lanes of a warp, with entry k = min(lane, 8) of C in ck
// (row-major). The FP32 steps run in every lane on the same values (the nine
// entries gathered by shuffles); the FP64 steps take one entry per lane. On
// true, lane k < 9 holds entry k of the rotation in rk. Returns false (in
// every lane) when C is not safely positive-determinant: the caller then
// takes the eigen-decomposition route, which also handles rank deficiency.
static __device__ bool polar_rotation_warp(double ck, int lane, double& rk) {
  const double nc2 = lane_sum9(ck * ck);  // |C|_F^2
  if (!(nc2 > 0.0) || !isfinite(nc2)) return false;
  const double s0 = (double)rsqrtf((float)nc2);
  const float xk = (float)(ck * s0);
  float Xf[9];  // |X|_F ~ 1 throughout
#pragma unroll
  for (int j = 0; j < 9; ++j) Xf[j] = __shfl_sync(FULL, xk, j);
  // The scale g only speeds the iteration up and the FP32 steps only have to
  // come within about 1e-6 of U V^T, so the reciprocal and the fourth root
  // are the SFU's approximations.
  bool converged32 = false;
  for (int it = 0; it < 40; ++it) {
    float cf[9];
    const float det = cof3(Xf, cf);
    if (!(det > 1e-6f)) return false;  // near rank 2 (or det < 0): the eigen route decides
    float idet;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(idet) : "f"(det));
    float x2[9], c2[9];
    for (int k = 0; k < 9; ++k) {
      cf[k] *= idet;
      x2[k] = Xf[k] * Xf[k];
      c2[k] = cf[k] * cf[k];
    }
    const float xx = ((x2[0] + x2[1]) + (x2[2] + x2[3])) + ((x2[4] + x2[5]) + (x2[6] + x2[7])) + x2[8];
    const float ii = ((c2[0] + c2[1]) + (c2[2] + c2[3])) + ((c2[4] + c2[5]) + (c2[6] + c2[7])) + c2[8];
    float ixx;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(ixx) : "f"(xx));
    const float r4 = rsqrt_fast(ii * ixx);  // |X|_F / |X^-T|_F
    const float g = rsqrt_fast(r4);         // (|X^-T|_F / |X|_F)^(1/2)
    const float a = 0.5f * g, b = 0.5f * r4 * g;  // 1/g = r4 * g
    float d2[9];
    for (int k = 0; k < 9; ++k) {
      const float xn = fmaf(a, Xf[k], b * cf[k]);
      d2[k] = (xn - Xf[k]) * (xn - Xf[k]);
      Xf[k] = xn;
    }
    const float change = ((d2[0] + d2[1]) + (d2[2] + d2[3])) + ((d2[4] + d2[5]) + (d2[6] + d2[7])) + d2[8];
    if (change < 1e-12f) {
      converged32 = true;
      break;
    }
  }
  // FP64 steps, entry k = (r, c) per lane; cofactor operands by shuffles
  const int k = lane < 9 ? lane : 8;
  const int r = k / 3, c = k - 3 * r;
  const int r1 = r == 2 ? 0 : r + 1, r2 = r == 0 ? 2 : r - 1;
  const int c1 = c == 2 ? 0 : c + 1, c2 = c == 0 ? 2 : c - 1;
  double x = (double)pick9(Xf, k);
  for (int it = 0; it < 8; ++it) {
    double det;
    const double cf = lane_cof3(x, r1, r2, c1, c2, det);
    if (!(det > 1e-9)) return false;
    const double h = 0.5 * rcp64(det);
    const double xn = fma(h, cf, 0.5 * x);
    if (converged32) {
      x = xn;
      break;
    }
    const double dd = (xn - x) * (xn - x);
    x = xn;
    if (lane_sum9(dd) < 1e-28) break;
  }
  // Newton's iteration keeps the singular vectors of its start, so its limit
  // is the polar factor of the FP32 iterate, whose rotation still carries the
  // FP32 steps' rounding (about 1e-9). One correction against C itself
  // removes it. With Q0 = x (orthogonal to FP64 precision) and C = Q H (H
  // symmetric positive definite), M = Q0^T C = R_d H, R_d = Q0^T Q =
  // exp([w]x); to first order in w, M - M^T = [w]x H + H [w]x =
  // [(tr H I - H) w]x with H = (M + M^T) / 2, so w solves
  // (tr H I - H) w = axial(M - M^T), and Q = Q0 (I + [w]x), whose row r is
  // q_r + q_r x w, up to an error of order |w|^2. C enters scaled to unit
  // Frobenius norm (w does not depend on the scale).
  {
    const double cs = ck * s0;
    const double m = __shfl_sync(FULL, x, r) * __shfl_sync(FULL, cs, c) +
                     __shfl_sync(FULL, x, 3 + r) * __shfl_sync(FULL, cs, 3 + c) +
                     __shfl_sync(FULL, x, 6 + r) * __shfl_sync(FULL, cs, 6 + c);
    const double trh = __shfl_sync(FULL, m, 0) + __shfl_sync(FULL, m, 4) + __shfl_sync(FULL, m, 8);
    const double a = (r == c ? trh : 0.0) - 0.5 * (m + __shfl_sync(FULL, m, 3 * c + r));
    double deta;
    const double cfa = lane_cof3(a, r1, r2, c1, c2, deta);
    if (deta > 1e-30) {
      // axial(M - M^T) = (m21 - m12, m02 - m20, m10 - m01); A = tr H I - H is
      // symmetric, so A^{-1} = cof(A) / det A; lane j < 3 takes w_j
      const double ax0 = __shfl_sync(FULL, m, 7) - __shfl_sync(FULL, m, 5);
      const double ax1 = __shfl_sync(FULL, m, 2) - __shfl_sync(FULL, m, 6);
      const double ax2 = __shfl_sync(FULL, m, 3) - __shfl_sync(FULL, m, 1);
      const int j = lane < 3 ? lane : 2;
      const double wj = (__shfl_sync(FULL, cfa, 3 * j) * ax0 + __shfl_sync(FULL, cfa, 3 * j + 1) * ax1 +
                         __shfl_sync(FULL, cfa, 3 * j + 2) * ax2) * rcp64(deta);
      const double w0 = __shfl_sync(FULL, wj, 0), w1 = __shfl_sync(FULL, wj, 1), w2 = __shfl_sync(FULL, wj, 2);
      const double wc1 = c1 == 0 ? w0 : (c1 == 1 ? w1 : w2), wc2 = c2 == 0 ? w0 : (c2 == 1 ? w1 : w2);
      // entry c of q_r x w: q_r[c + 1] w[c + 2] - q_r[c + 2] w[c + 1]
      x += __shfl_sync(FULL, x, 3 * r + c1) * wc2 - __shfl_sync(FULL, x, 3 * r + c2) * wc1;
    }
  }
  rk = x;
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

constexpr int EPI_BS_MIN = 128;  // fewest threads of a block that calls rigid_step_block

// Shared values between the phases of the fit.
struct FitShared {
  double Rp[9], tp[3];  // R', t' of this iteration
};

// Called by every thread of the block that finishes an iteration (Eqs. 14,
// 16 and Algorithm 2's composition and stop test), with the state in shared
// memory; needs at least 44 threads. FP64 instructions cost a warp about 64
// cycles each however few lanes are active, so the matrices of the fit are
// spread over the lanes of warp 0, one entry per lane:
//  1. lane k forms entry k of C from the reductions; the warp takes R'
//     (polar route; the eigen route, or R' = I for a degenerate C, in every
//     lane when that fails) and lanes 0-2 take t';
//  2. lanes 0-11 of warp 0 compose [R | t] entry by entry with the
//     convergence terms, which they add by shuffles; lanes 0-11 of warp 1 take
//     the rigid-velocity coefficients at the same time;
//  3. warp 0 updates the flags, the history and the FP32 copies, one entry
//     per lane.
// red: the NRED reduced values (shared memory); ds: the state (shared
// memory), updated in place and visible to the whole block on return.
static __device__ void rigid_step_smem(const double* red, int64_t M, DevState* ds, const EpiParams& ep,
                                       double* traj, unsigned long long inter_add) {
  __shared__ FitShared f;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  if (tid < 32) {
    // C = S + Dy - M (ybar + mud) ybar^T: S = sum yc yc^T (symmetric: xx, xy,
    // xz, yy, yz, zz in red[6..11]), Dy = sum d yc^T, ybar the mean of the
    // centred template (~0), mud the mean displacement
    const int k = lane < 9 ? lane : 8;
    const int r = k / 3, c = k - 3 * r;
    const int lo = r < c ? r : c, hi = r < c ? c : r;
    const int si = 6 + (lo == 0 ? hi : (lo == 1 ? 2 + hi : 5));
    const double Md = (double)M;
    const double ybar_r = red[r] * ep.inv_M, mud_r = red[3 + r] * ep.inv_M, ybar_c = red[c] * ep.inv_M;
    const double ck = red[si] + red[12 + k] - Md * (ybar_r + mud_r) * ybar_c;
    double rk = 0.0;
    bool ok;
    if (ep.dim == 2) {
      double C[9], Rp[9];
#pragma unroll
      for (int j = 0; j < 9; ++j) C[j] = __shfl_sync(FULL, ck, j);
      ok = planar_rotation(C, Rp);
      if (ok) rk = pick9(Rp, k);
    } else {
      ok = polar_rotation_warp(ck, lane, rk);
      if (!ok) {
        double C[9], Rp[9];
#pragma unroll
        for (int j = 0; j < 9; ++j) C[j] = __shfl_sync(FULL, ck, j);
        ok = rigid_rotation(C, Rp);
        if (ok) rk = pick9(Rp, k);
      }
    }
    if (!ok) {
      rk = (k % 4 == 0) ? 1.0 : 0.0;
      if (lane == 0) ds->degenerate += 1;
    }
    if (lane < 9) f.Rp[lane] = rk;
    // t' = mu_Y + mu_D - R' mu_Y, mu_Y = muf + ybar (muf is the FP32 centre
    // the kernels subtracted)
    const int q3 = lane < 3 ? lane : 2;
    const double muy = (double)ds->muf[q3] + red[q3] * ep.inv_M;
    const double mu0 = __shfl_sync(FULL, muy, 0), mu1 = __shfl_sync(FULL, muy, 1),
                 mu2 = __shfl_sync(FULL, muy, 2);
    __syncwarp();
    if (lane < 3) {
      const double mud = red[3 + lane] * ep.inv_M;
      f.tp[lane] = muy + mud - (f.Rp[3 * lane] * mu0 + f.Rp[3 * lane + 1] * mu1 + f.Rp[3 * lane + 2] * mu2);
    }
  }
  __syncthreads();
  const int k_it = ds->iter;
  if (tid < 32) {
    // [R | t] <- [R'R | R't + t'], entry q per lane
    const int q = lane < 12 ? lane : 11;
    double v;
    if (q < 9) {
      const int r = q / 3, c = q % 3;
      v = f.Rp[3 * r] * ds->R[c] + f.Rp[3 * r + 1] * ds->R[3 + c] + f.Rp[3 * r + 2] * ds->R[6 + c];
    } else {
      const int r = q - 9;
      v = f.Rp[3 * r] * ds->t[0] + f.Rp[3 * r + 1] * ds->t[1] + f.Rp[3 * r + 2] * ds->t[2] + f.tp[r];
    }
    const double e = (v - ds->Tm2[q]) * (v - ds->Tm2[q]);
    // |T_k - T_{k-2}|_F^2 = ((e0 + e1) + (e2 + e3)) + ((e4 + e5) + (e6 + e7)) + ((e8 + e9) + (e10 + e11))
    const double b1 = e + __shfl_down_sync(FULL, e, 1);
    const double b2 = b1 + __shfl_down_sync(FULL, b1, 2);
    const double b3 = b2 + __shfl_down_sync(FULL, b2, 4);
    const double d2 = b3 + __shfl_sync(FULL, b2, 8);  // lane 0
    const bool finite = __all_sync(FULL, lane >= 12 || isfinite(v));
    __syncwarp();  // every lane has read R, t and the history before they change
    if (lane == 0) {
      if (k_it >= 2) {
        ds->last_conv = d2;
        if (ep.conv_tol > 0 && d2 <= ep.conv_tol) {
          ds->done = 1;
          ds->converged = 1;
        }
      } else {
        ds->last_conv = -1.0;
      }
      if (!finite) {
        ds->status |= 2;
        ds->done = 1;
      }
      ds->interactions += inter_add;
      ds->iter = k_it + 1;
      if (ep.max_iter > 0 && k_it + 1 >= ep.max_iter) ds->done = 1;
    }
    if (lane < 12) {
      ds->Tm2[lane] = ds->Tm1[lane];
      ds->Tm1[lane] = v;
      if (lane < 9) {
        ds->R[lane] = v;
        ds->Rf[lane] = (float)v;
      } else {
        ds->t[lane - 9] = v;
        ds->tf[lane - 9] = (float)v;
      }
      if (traj && k_it < ep.max_traj) traj[12 * (int64_t)k_it + lane] = v;
    } else if (lane < 15) {
      ds->netF[lane - 12] = red[21 + lane - 12];
    } else if (lane < 18) {
      ds->torque[lane - 15] = red[24 + lane - 15];
    }
    __syncwarp();
    // the FP32 centre that the kernels subtract (any value near the
    // template's centroid serves, as long as the fit adds back the same one)
    if (lane < 3) {
      const float m0 = (float)ds->mu0[0], m1 = (float)ds->mu0[1], m2 = (float)ds->mu0[2];
      const int r = lane;
      ds->muf[r] = fmaf(ds->Rf[3 * r], m0, fmaf(ds->Rf[3 * r + 1], m1, fmaf(ds->Rf[3 * r + 2], m2, ds->tf[r])));
    }
  } else if (tid < 44) {
    // rigid velocity of the next iteration: v = (y_new - y_old)/dt with
    // y_old = R'^T (y_new - t'), i.e. v = (I - R'^T)/dt y_new + R'^T t'/dt
    const double idt = ep.inv_dt;
    const int q = tid - 32;
    if (q < 9) {
      const int r = q / 3, c = q % 3;
      ds->A[q] = (float)(((r == c ? 1.0 : 0.0) - f.Rp[3 * c + r]) * idt);
    } else {
      const int r = q - 9;
      ds->b[r] = (float)((f.Rp[r] * f.tp[0] + f.Rp[3 + r] * f.tp[1] + f.Rp[6 + r] * f.tp[2]) * idt);
    }
  }
  __syncthreads();
}

// rigid_step_smem for a block whose state lives in global memory (ds_g): the
// block copies the state into shared memory (8 bytes per thread, one round
// trip; one thread reading the fields in global memory would wait behind its
// own earlier stores to the same struct), takes the step there and copies the
// state back.
static __device__ void rigid_step_block(const double* red, int64_t M, DevState* ds_g, const EpiParams& ep,
                                        double* traj, unsigned long long inter_add) {
  static_assert(sizeof(DevState) % sizeof(unsigned long long) == 0, "state copied in 8-byte words");
  constexpr int NW = (int)(sizeof(DevState) / sizeof(unsigned long long));
  static_assert(NW <= EPI_BS_MIN, "one word per thread");
  __shared__ DevState s_state;
  unsigned long long* sw = reinterpret_cast<unsigned long long*>(&s_state);
  unsigned long long* gw = reinterpret_cast<unsigned long long*>(ds_g);
  const int tid = threadIdx.x;
  if (tid < NW) sw[tid] = __ldcg(gw + tid);
  __syncthreads();
  rigid_step_smem(red, M, &s_state, ep, traj, inter_add);
  if (tid < NW) gw[tid] = sw[tid];
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

// Eq. 9 with the dissipative force of Eq. 7, v' = v + dt (a - eta v / m_Y),
// and Eq. 10, d = dt v', for template point i with acceleration a = G * sum
// (sx, sy, sz). Adds the point's 27 reduction terms to r: centred position
// yc, d, yc yc^T (6), d yc^T (9), force m_Y a, torque yc x m_Y a.
__device__ __forceinline__ void epi_ode(int64_t i, float4 y0, float sx, float sy, float sz,
                                        float4* __restrict__ V, const EpiParams& ep, const EpiCtx& c,
                                        float (&r)[NRED]);

// Template point i with the force given as the compensated sum of S partial
// sums (the all-pairs source splits, or the batch kernels' frontier cells).
// `live`: bit s set for the slots to add (all S slots when no mask is kept);
// the others are exact zeros, and adding a zero never changes a compensated
// sum, so the result is the same as adding all S slots in order.
__device__ __forceinline__ void epi_point(int64_t i, const float4* __restrict__ Y0,
                                          const float4* __restrict__ hi, const float4* __restrict__ lo,
                                          int S, int64_t M, float4* __restrict__ V,
                                          const EpiParams& ep, const EpiCtx& c, float (&r)[NRED],
                                          unsigned long long live = ~0ull) {
  const float4 y0 = Y0[i];
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
  epi_ode(i, y0, ahx + alx, ahy + aly, ahz + alz, V, ep, c, r);
}

// Template point i with the force given as exact fixed-point sums (three
// planes of M, value = integer * unscale): read, rounded once to FP32, and
// cleared for the next launch.
__device__ __forceinline__ void epi_point_fixed(int64_t i, const float4* __restrict__ Y0,
                                                long long* __restrict__ acc, float unscale, int64_t M,
                                                float4* __restrict__ V, const EpiParams& ep,
                                                const EpiCtx& c, float (&r)[NRED]) {
  const float4 y0 = Y0[i];
  const long long ix = acc[i], iy = acc[M + i], iz = acc[2 * M + i];
  acc[i] = 0;
  acc[M + i] = 0;
  acc[2 * M + i] = 0;
  epi_ode(i, y0, __ll2float_rn(ix) * unscale, __ll2float_rn(iy) * unscale, __ll2float_rn(iz) * unscale, V,
          ep, c, r);
}

__device__ __forceinline__ void epi_ode(int64_t i, float4 y0, float sx, float sy, float sz,
                                        float4* __restrict__ V, const EpiParams& ep, const EpiCtx& c,
                                        float (&r)[NRED]) {
  const float3 y = place(c.xf, y0);
  const float cx = y.x - c.mu[0], cy = y.y - c.mu[1], cz = y.z - c.mu[2];
  const float ax = ep.G * sx, ay = ep.G * sy, az = ep.G * sz;
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
// thread of the block must call it. Each warp sum is converted to FP64 by a
// thread of its own (an FP64 instruction costs the warp the same for one
// lane as for 32), and NRED lanes add the warp sums at once.
__device__ __forceinline__ void epi_block_partial(float (&r)[NRED], double* __restrict__ out) {
  constexpr int NWB = EPI_BS / 32;
  __shared__ float s_wf[NWB][NRED];
  __shared__ double s_w[NWB][NRED];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NRED; ++k)
    for (int off = 16; off > 0; off >>= 1) r[k] += __shfl_down_sync(FULL, r[k], off);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NRED; ++k) s_wf[w][k] = r[k];
  __syncthreads();
  if (threadIdx.x < NWB * NRED) {
    const int ww = threadIdx.x / NRED, k = threadIdx.x - ww * NRED;
    s_w[ww][k] = (double)s_wf[ww][k];
  }
  __syncthreads();
  if (threadIdx.x < NRED) {
    double acc = s_w[0][threadIdx.x];
    for (int ww = 1; ww < NWB; ++ww) acc += s_w[ww][threadIdx.x];
    out[threadIdx.x] = acc;
  }
}

// FP64 sum of nblocks x NRED partials in a fixed order, by the whole block:
// thread t < 8 NRED adds value t % NRED over blocks t / NRED, + 8, ...;
// NRED threads then add the strands (at most 8) into s_red (shared, NRED
// doubles). FP64 adds are scarce on this GPU, so no FP64 warp shuffles are
// used and no zero is added.
__device__ __forceinline__ void epi_last_reduce(const double* partials, int nblocks, double* s_red) {
  __shared__ double s_strand[8][NRED];
  if (threadIdx.x < 8 * NRED) {
    const int k = threadIdx.x % NRED, j = threadIdx.x / NRED;
    if (j < nblocks) {
      double acc = __ldcg(&partials[(int64_t)j * NRED + k]);
      for (int b = j + 8; b < nblocks; b += 8) acc += __ldcg(&partials[(int64_t)b * NRED + k]);
      s_strand[j][k] = acc;
    }
  }
  __syncthreads();
  if (threadIdx.x < NRED) {
    double acc = s_strand[0][threadIdx.x];
    const int ns = nblocks < 8 ? nblocks : 8;
    for (int j = 1; j < ns; ++j) acc += s_strand[j][threadIdx.x];
    s_red[threadIdx.x] = acc;
  }
  __syncthreads();
}

}  // namespace fga
