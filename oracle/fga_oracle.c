/*
 * FP64 CPU oracle of the Fast Gravitational Approach (FGA) hot path
 * (Ali, Kahraman, Golyanik, Stricker: "Fast Gravitational Approach for Rigid
 * Point Set Registration with Ordinary Differential Equations", arXiv 2009.14005).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, obviously-correct reference
 * that the CUDA library is checked against. Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg load it. The library never calls
 * it and shares no code with it.
 *
 * Everything is plain double precision, loops in index order, one function per
 * step of the paper:
 *   orc_normalize / orc_denormalize  Appendix, Eqs. A.1-A.3 (and the derivation
 *                                    of dnorm(t) that follows them)
 *   orc_masses_niv                   Sec. IV-F.2, Eq. 18 (NIV measure)
 *   orc_masses_knn                   Sec. IV-F (point masses from a per-point
 *                                    feature): inverse local density from the
 *                                    distance to the k-th nearest neighbour
 *   orc_masses_rbf                   Sec. IV-F.1, Eq. 17 (RBF mass interpolant);
 *                                    with the NIV weights, Eq. 19 (SPM) is
 *                                    their point-wise product
 *   orc_direct_acc                   Sec. IV-C, Eq. 6 (all-pairs force)
 *   orc_tree_build                   Sec. IV-E, Algorithm 1 (BH tree)
 *   orc_bh_acc                       Sec. IV-E, Eq. 15 and BHForce in Algorithm 2
 *   orc_ode_step                     Eqs. 7-10 (damped velocity, displacement)
 *   orc_kabsch                       Sec. IV-D, Eqs. 14 and 16
 *   orc_register                     Algorithm 2 (the FGA loop)
 *
 * Readings of passages that the paper leaves open are marked "Reading".
 * OpenMP only splits independent template points over threads; the
 * arithmetic of each point is the same whatever the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double G, eps, eta, dt, theta;
    int max_iter;
    double conv_tol;     /* <= 0: run exactly max_iter iterations */
    int method;          /* 0 = all-pairs sum (Eq. 6), 1 = Barnes-Hut */
    int velocity_mode;   /* 0 = unconstrained velocities kept (Eq. 9),
                            1 = velocities replaced by the rigid motion   */
    int max_depth;       /* depth limit of the BH tree (paper: 20) */
    int dim;             /* D = 3, or D = 2 for clouds in the plane z = 0:
                            the tree is then the quadtree (no z split), and the
                            rigid fit of Eq. 14 is the 2 x 2 one */
} orc_params;

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Appendix A: normalisation into [a, b] and de-normalisation of t           */
/* ------------------------------------------------------------------------ */

/* A.1: means of X and Y; A.2: global scalar min l and max r over all
 * coordinates of both centred clouds; A.3: X^ = (X - Xbar - l)(b-a)/(r-l) + a.
 * info = {Xbar[3], Ybar[3], l, s} with s = (b-a)/(r-l).
 * Returns 0, or -1 if r == l (every coordinate of both centred clouds equal). */
int orc_normalize(const double* X, long N, const double* Y, long M, double a, double b,
                  double* Xn, double* Yn, double info[8]) {
    double xb[3] = {0, 0, 0}, yb[3] = {0, 0, 0};
    for (long j = 0; j < N; ++j)
        for (int k = 0; k < 3; ++k) xb[k] += X[3 * j + k];
    for (long i = 0; i < M; ++i)
        for (int k = 0; k < 3; ++k) yb[k] += Y[3 * i + k];
    for (int k = 0; k < 3; ++k) { xb[k] /= (double)N; yb[k] /= (double)M; }
    double l = INFINITY, r = -INFINITY;
    for (long j = 0; j < N; ++j)
        for (int k = 0; k < 3; ++k) {
            double v = X[3 * j + k] - xb[k];
            if (v < l) l = v;
            if (v > r) r = v;
        }
    for (long i = 0; i < M; ++i)
        for (int k = 0; k < 3; ++k) {
            double v = Y[3 * i + k] - yb[k];
            if (v < l) l = v;
            if (v > r) r = v;
        }
    if (!(r > l)) return -1;
    double s = (b - a) / (r - l);
    for (long j = 0; j < N; ++j)
        for (int k = 0; k < 3; ++k) Xn[3 * j + k] = (X[3 * j + k] - xb[k] - l) * s + a;
    for (long i = 0; i < M; ++i)
        for (int k = 0; k < 3; ++k) Yn[3 * i + k] = (Y[3 * i + k] - yb[k] - l) * s + a;
    for (int k = 0; k < 3; ++k) { info[k] = xb[k]; info[3 + k] = yb[k]; }
    info[6] = l;
    info[7] = s;
    return 0;
}

/* Reading of the Appendix's dnorm(t): substituting A.3 for both clouds into
 * R Y^ + t = X^ and solving for X gives X = R Y + t_orig with
 *   t_orig = Xbar - R Ybar + l (1 - R 1) + (R a1 + t - a1) / s,
 * where 1 = (1,1,1). The rotation is unchanged by the isotropic scaling. */
void orc_denormalize(const double R[9], const double t[3], const double info[8], double a,
                     double t_out[3]) {
    const double* xb = info;
    const double* yb = info + 3;
    double l = info[6], s = info[7];
    for (int r = 0; r < 3; ++r) {
        double rybar = 0, rsum = 0;
        for (int c = 0; c < 3; ++c) {
            rybar += R[3 * r + c] * yb[c];
            rsum += R[3 * r + c];
        }
        t_out[r] = xb[r] - rybar + l * (1.0 - rsum) + (a * rsum + t[r] - a) / s;
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. IV-F.2, Eq. 18: normalised intrinsic volume (NIV) masses             */
/* ------------------------------------------------------------------------ */

/* Quadrature of the covered fraction (a reading: the paper does not say how
 * the volume of the union of balls is obtained). Along the cell's last axis
 * (z in 3D, y in 2D) the union is taken exactly: every ball that reaches a
 * line through the cell cuts it in a chord, and the covered length of the line
 * is the length of the union of those chords, clipped to the cell. The other
 * axes are sampled by the midpoint rule: NIV_COLS x NIV_COLS lines per 3D cell,
 * NIV_STRIPS lines per 2D cell. Measured against closed forms (one ball, two
 * overlapping balls, a ball cut by a cell face) the fraction is within 3e-3
 * (3D) and 1.1e-4 (2D) of the exact one. */
#define NIV_COLS 64
#define NIV_STRIPS 1024

typedef struct { double lo, hi; } orc_chord;

static int orc_chord_cmp(const void* pa, const void* pb) {
    const orc_chord* x = (const orc_chord*)pa;
    const orc_chord* y = (const orc_chord*)pb;
    return x->lo < y->lo ? -1 : (x->lo > y->lo ? 1 : 0);
}

/* Length of the union of k chords: sorted by their lower ends, swept once. */
static double orc_union_length(orc_chord* c, long k) {
    if (k == 0) return 0.0;
    qsort(c, (size_t)k, sizeof(orc_chord), orc_chord_cmp);
    double len = 0.0, s = c[0].lo, e = c[0].hi;
    for (long q = 1; q < k; ++q) {
        if (c[q].lo <= e) {
            if (c[q].hi > e) e = c[q].hi;
        } else {
            len += e - s;
            s = c[q].lo;
            e = c[q].hi;
        }
    }
    return len + (e - s);
}

/* Reading of the lattice: lattice^D equal cubes over the normalised domain
 * [a, b]^D, cell side h = (b - a) / lattice. A point's cell along each axis is
 * floor((x - a) / h) clamped to [0, lattice - 1], and its ball is centred at
 * the point clamped to [a, b] (so it always touches its own cell). The ball
 * radius of Eq. 18 is (b - a) / (2 d lattice) = h / (2 D), d read as the
 * dimension D. The covered fraction of a cell is V(union of its points'
 * balls, inside the cell) / V(cell) (Eq. 18 and the caption of the NIV
 * figure: the part of the cell occupied by the balls inside it). A point's
 * weight is 1 / fraction of its cell (Eq. 18; the normalising integral is a
 * common factor that cancels), and the weights are scaled to sum to `total`.
 * dim 2 uses x, y: discs of radius h / 4 in square cells.
 *
 * orc_niv_fractions writes the covered fraction of every cell to frac
 * (lattice^D entries, 0 for empty cells, indexed (cz * lattice + cy) *
 * lattice + cx) and each point's cell to cell (n entries). The test-suite
 * checks these fractions against closed forms. Returns 0, -1 for bad
 * arguments, -2 if memory ran out. */
int orc_niv_fractions(const double* P, long n, int dim, int lattice, double a, double b,
                      double* frac, long* cell) {
    if (n <= 0 || lattice <= 0 || !(b > a) || (dim != 2 && dim != 3)) return -1;
    long ncell = dim == 3 ? (long)lattice * lattice * lattice : (long)lattice * lattice;
    long* count = (long*)calloc((size_t)ncell + 1, sizeof(long));
    long* order = (long*)malloc((size_t)n * sizeof(long));
    long* fill = (long*)malloc((size_t)ncell * sizeof(long));
    if (!count || !order || !fill) {
        free(count); free(order); free(fill);
        return -2;
    }
    for (long c = 0; c < ncell; ++c) frac[c] = 0.0;
    const double h = (b - a) / (double)lattice;
    for (long i = 0; i < n; ++i) {
        long c[3] = {0, 0, 0};
        for (int k = 0; k < dim; ++k) {
            double q = floor((P[3 * i + k] - a) / h);
            if (q > lattice - 1) q = lattice - 1;
            if (q < 0) q = 0;
            c[k] = (long)q;
        }
        cell[i] = (c[2] * lattice + c[1]) * lattice + c[0];
        count[cell[i] + 1] += 1;
    }
    /* points grouped by cell, in index order within a cell */
    for (long c = 0; c < ncell; ++c) count[c + 1] += count[c];
    memcpy(fill, count, (size_t)ncell * sizeof(long));
    for (long i = 0; i < n; ++i) order[fill[cell[i]]++] = i;
    free(fill);
    const double rad = (b - a) / (2.0 * (double)dim * (double)lattice);
    const double rr = rad * rad;
    const int q = dim == 3 ? NIV_COLS : NIV_STRIPS;
    const double dlt = h / (double)q;
    const long nlines = dim == 3 ? (long)q * q : (long)q;
    int fail = 0;
#pragma omp parallel
    {
        orc_chord* ch = NULL;
        long cap = 0;
#pragma omp for schedule(dynamic, 1)
        for (long c = 0; c < ncell; ++c) {
            long first = count[c], nc = count[c + 1] - first;
            if (nc == 0) continue;
            if (nc > cap) {
                orc_chord* t = (orc_chord*)realloc(ch, (size_t)nc * sizeof(orc_chord));
                if (!t) {
#pragma omp atomic write
                    fail = 1;
                    continue;
                }
                ch = t;
                cap = nc;
            }
            long cx = c % lattice, cy = (c / lattice) % lattice, cz = c / ((long)lattice * lattice);
            double lox = a + (double)cx * h, loy = a + (double)cy * h, loz = a + (double)cz * h;
            /* the chord axis: z in 3D, y in 2D */
            double clo = dim == 3 ? loz : loy, chi = clo + h;
            double covered = 0.0;
            for (long ln = 0; ln < nlines; ++ln) {
                double u = lox + ((double)(ln % q) + 0.5) * dlt;              /* x of the line */
                double v = dim == 3 ? loy + ((double)(ln / q) + 0.5) * dlt : 0; /* y (3D)      */
                long k = 0;
                for (long t = 0; t < nc; ++t) {
                    const double* p = P + 3 * order[first + t];
                    double px = fmin(fmax(p[0], a), b), py = fmin(fmax(p[1], a), b);
                    double d2, zc;
                    if (dim == 3) {
                        double pz = fmin(fmax(p[2], a), b);
                        d2 = (u - px) * (u - px) + (v - py) * (v - py);
                        zc = pz;
                    } else {
                        d2 = (u - px) * (u - px);
                        zc = py;
                    }
                    if (d2 >= rr) continue;
                    double w = sqrt(rr - d2);
                    double lo = zc - w, hi = zc + w;
                    if (lo < clo) lo = clo;
                    if (hi > chi) hi = chi;
                    if (hi > lo) { ch[k].lo = lo; ch[k].hi = hi; ++k; }
                }
                covered += orc_union_length(ch, k);
            }
            frac[c] = covered / ((double)nlines * h);
        }
        free(ch);
    }
    free(count);
    free(order);
    return fail ? -2 : 0;
}

/* Eq. 18 masses: 1 / (covered fraction of the point's cell), scaled to sum to
 * `total`. */
int orc_masses_niv_d(const double* P, long n, int dim, int lattice, double a, double b, double total,
                     double* m_out) {
    if (n <= 0 || lattice <= 0 || !(b > a) || (dim != 2 && dim != 3)) return -1;
    long ncell = dim == 3 ? (long)lattice * lattice * lattice : (long)lattice * lattice;
    double* frac = (double*)malloc((size_t)ncell * sizeof(double));
    long* cell = (long*)malloc((size_t)n * sizeof(long));
    if (!frac || !cell) { free(frac); free(cell); return -2; }
    int rc = orc_niv_fractions(P, n, dim, lattice, a, b, frac, cell);
    if (rc) { free(frac); free(cell); return rc; }
    double wsum = 0;
    for (long i = 0; i < n; ++i) {
        m_out[i] = 1.0 / frac[cell[i]];
        wsum += m_out[i];
    }
    for (long i = 0; i < n; ++i) m_out[i] = total * m_out[i] / wsum;
    free(frac);
    free(cell);
    return 0;
}

int orc_masses_niv(const double* P, long n, int lattice, double a, double b, double total,
                   double* m_out) {
    return orc_masses_niv_d(P, n, 3, lattice, a, b, total, m_out);
}

/* ------------------------------------------------------------------------ */
/* Inverse-density masses from the k-th nearest neighbour                     */
/* ------------------------------------------------------------------------ */

/* Reading (a smooth-particle mass from the k nearest neighbours): the local
 * density at P_i is k points per ball reaching its k-th nearest other point,
 * of radius r_k(i); the mass is inversely proportional to it, m_i ~ r_k(i)^D
 * (D = dim, the ball's volume up to a constant), r_k floored at
 * r_min = 1e-6 (b - a) so that repeated points keep a positive mass. Scaled
 * to sum to `total`. Brute force: every other point, k smallest squared
 * distances kept sorted. dim 2 uses the x, y components. */
int orc_masses_knn(const double* P, long n, int k, int dim, double a, double b, double total,
                   double* m_out) {
    if (n <= (long)k || k < 1 || k > 64 || (dim != 2 && dim != 3) || !(b > a)) return -1;
    const double rmin = 1e-6 * (b - a);
    double wsum = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : wsum)
    for (long i = 0; i < n; ++i) {
        double best[64];
        int have = 0;
        for (long j = 0; j < n; ++j) {
            if (j == i) continue;
            double d2 = 0;
            for (int c = 0; c < dim; ++c) {
                double d = P[3 * j + c] - P[3 * i + c];
                d2 += d * d;
            }
            if (have < k) {
                int q = have++;
                while (q > 0 && best[q - 1] > d2) { best[q] = best[q - 1]; --q; }
                best[q] = d2;
            } else if (d2 < best[k - 1]) {
                int q = k - 1;
                while (q > 0 && best[q - 1] > d2) { best[q] = best[q - 1]; --q; }
                best[q] = d2;
            }
        }
        double r = sqrt(best[k - 1]);
        if (r < rmin) r = rmin;
        m_out[i] = dim == 3 ? r * r * r : r * r;
        wsum += m_out[i];
    }
    for (long i = 0; i < n; ++i) m_out[i] = total * m_out[i] / wsum;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sec. IV-F.1, Eq. 17: RBF mass interpolant from landmarks                  */
/* ------------------------------------------------------------------------ */

/* B(P_i) = sum_c lambda_c Phi(|P_i - P_c|), Phi(s) = exp(-s^2 / sigma^2), over
 * the m landmarks c = idx[0..m-1] (Eq. 17; B = 1 everywhere when m = 0).
 * Reading: Eq. 17 writes the coefficients lambda_{i c}; they are those of the
 * standard RBF interpolant, one per landmark, fixed by collocation at the
 * landmarks: sum_c' Phi(|P_c - P_c'|) lambda_c' = w_c with w_c = 1, the
 * "strong weight" the paper gives landmarks. sigma is the kernel width (the
 * paper gives none). B is then clamped below at `floor` (> 0) so that every
 * mass stays positive far from the landmarks.
 * The m x m system (symmetric positive definite for distinct landmarks) is
 * solved by Cholesky factorisation in index order. Returns 0, -1 for bad
 * arguments, -2 when the collocation matrix is not positive definite
 * (repeated landmarks). */
int orc_masses_rbf(const double* P, long n, const long* idx, int m, double sigma, double floor_v,
                   double* B_out) {
    if (n <= 0 || m < 0 || !(sigma > 0) || !(floor_v > 0)) return -1;
    for (int c = 0; c < m; ++c)
        if (idx[c] < 0 || idx[c] >= n) return -1;
    if (m == 0) {
        for (long i = 0; i < n; ++i) B_out[i] = 1.0;
        return 0;
    }
    double* A = (double*)malloc((size_t)m * m * sizeof(double));
    double* lam = (double*)malloc((size_t)m * sizeof(double));
    if (!A || !lam) { free(A); free(lam); return -2; }
    const double is2 = 1.0 / (sigma * sigma);
    for (int r = 0; r < m; ++r)
        for (int c = 0; c < m; ++c) {
            double d2 = 0;
            for (int k = 0; k < 3; ++k) {
                double d = P[3 * idx[r] + k] - P[3 * idx[c] + k];
                d2 += d * d;
            }
            A[r * m + c] = exp(-d2 * is2);
        }
    /* Cholesky A = L L^T (L overwrites the lower triangle) */
    for (int j = 0; j < m; ++j) {
        double s = A[j * m + j];
        for (int k = 0; k < j; ++k) s -= A[j * m + k] * A[j * m + k];
        if (!(s > 0)) { free(A); free(lam); return -2; }
        const double ljj = sqrt(s);
        A[j * m + j] = ljj;
        for (int i = j + 1; i < m; ++i) {
            double t = A[i * m + j];
            for (int k = 0; k < j; ++k) t -= A[i * m + k] * A[j * m + k];
            A[i * m + j] = t / ljj;
        }
    }
    /* L z = w (w = 1), then L^T lambda = z */
    for (int i = 0; i < m; ++i) {
        double t = 1.0;
        for (int k = 0; k < i; ++k) t -= A[i * m + k] * lam[k];
        lam[i] = t / A[i * m + i];
    }
    for (int i = m - 1; i >= 0; --i) {
        double t = lam[i];
        for (int k = i + 1; k < m; ++k) t -= A[k * m + i] * lam[k];
        lam[i] = t / A[i * m + i];
    }
    for (long i = 0; i < n; ++i) {
        double b = 0;
        for (int c = 0; c < m; ++c) {
            double d2 = 0;
            for (int k = 0; k < 3; ++k) {
                double d = P[3 * i + k] - P[3 * idx[c] + k];
                d2 += d * d;
            }
            b += lam[c] * exp(-d2 * is2);
        }
        B_out[i] = b > floor_v ? b : floor_v;
    }
    free(A);
    free(lam);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sec. IV-C, Eq. 6: gravitational force on template point i from all X_j    */
/* ------------------------------------------------------------------------ */

/* acc[i] = G sum_j m_j (X_j - Y_i) / (|X_j - Y_i|^2 + eps^2)^(3/2).
 * This is Eq. 6 divided by m_Yi (F_Yi / m_Yi): the template mass cancels in
 * Eq. 9 for the gravity term. absacc[i] (optional) is the same sum of the
 * term magnitudes, the natural scale of rounding error in the sum. */
void orc_direct_acc(const double* X, const double* mX, long N, const double* Y, long M, double G,
                    double eps, double* acc, double* absacc) {
    double e2 = eps * eps;
#pragma omp parallel for schedule(static)
    for (long i = 0; i < M; ++i) {
        double ax = 0, ay = 0, az = 0, aa = 0;
        for (long j = 0; j < N; ++j) {
            double dx = X[3 * j] - Y[3 * i];
            double dy = X[3 * j + 1] - Y[3 * i + 1];
            double dz = X[3 * j + 2] - Y[3 * i + 2];
            double d2 = dx * dx + dy * dy + dz * dz;
            double w = mX[j] / pow(d2 + e2, 1.5);
            ax += w * dx;
            ay += w * dy;
            az += w * dz;
            aa += w * sqrt(d2);
        }
        acc[3 * i] = G * ax;
        acc[3 * i + 1] = G * ay;
        acc[3 * i + 2] = G * az;
        if (absacc) absacc[i] = G * aa;
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. IV-E, Algorithm 1: Barnes-Hut tree on X                              */
/* ------------------------------------------------------------------------ */

typedef struct onode {
    double bmin[3], bmax[3]; /* cell box */
    double l;                /* |bmax - bmin|_2 (Algorithm 1) */
    double mass, com[3];
    int depth;
    long cell[3];            /* integer cell coordinates at this depth */
    long n;                  /* points inside */
    long* idx;               /* point indices (owned by leaves only) */
    int nchild;
    struct onode* child[8];  /* non-empty children in octant order */
} onode;

typedef struct {
    onode* root;
    const double* X;         /* not owned */
    double* Xc;              /* owned copy of X (n x 3) */
    double* m;               /* owned copy of the masses */
    long N;
    int max_depth;
} otree;

/* Algorithm 1, CreateChild: a cell holding more than one point and lying above
 * the depth limit is split at its box midpoint o = Xmin + (Xmax - Xmin)/2 into
 * 2^3 boxes; a point goes to the upper half along an axis iff its coordinate
 * is >= o there. Reading: an axis whose box has zero extent is not split (all
 * points take the lower half). Every non-empty cell gets l, mass and CoM. */
static onode* create_child(otree* T, long* idx, long n, const double bmin[3], const double bmax[3],
                           int depth, const long cell[3]) {
    onode* nd = (onode*)calloc(1, sizeof(onode));
    for (int k = 0; k < 3; ++k) {
        nd->bmin[k] = bmin[k];
        nd->bmax[k] = bmax[k];
        nd->cell[k] = cell[k];
    }
    nd->depth = depth;
    nd->n = n;
    double d2 = 0;
    for (int k = 0; k < 3; ++k) d2 += (bmax[k] - bmin[k]) * (bmax[k] - bmin[k]);
    nd->l = sqrt(d2);
    double ms = 0, cx = 0, cy = 0, cz = 0;
    for (long q = 0; q < n; ++q) {
        long j = idx[q];
        ms += T->m[j];
        cx += T->m[j] * T->Xc[3 * j];
        cy += T->m[j] * T->Xc[3 * j + 1];
        cz += T->m[j] * T->Xc[3 * j + 2];
    }
    nd->mass = ms;
    if (ms > 0) {
        nd->com[0] = cx / ms;
        nd->com[1] = cy / ms;
        nd->com[2] = cz / ms;
    } else { /* massless cell: its force is zero whatever the CoM; use the mean */
        double sx = 0, sy = 0, sz = 0;
        for (long q = 0; q < n; ++q) {
            sx += T->Xc[3 * idx[q]];
            sy += T->Xc[3 * idx[q] + 1];
            sz += T->Xc[3 * idx[q] + 2];
        }
        nd->com[0] = sx / n;
        nd->com[1] = sy / n;
        nd->com[2] = sz / n;
    }
    if (n > 1 && depth < T->max_depth) {
        double o[3];
        for (int k = 0; k < 3; ++k) o[k] = bmin[k] + (bmax[k] - bmin[k]) / 2.0;
        long* part = (long*)malloc((size_t)n * sizeof(long));
        long cnt[8] = {0};
        int* oct = (int*)malloc((size_t)n * sizeof(int));
        for (long q = 0; q < n; ++q) {
            long j = idx[q];
            int c = 0;
            for (int k = 0; k < 3; ++k)
                if (bmax[k] > bmin[k] && T->Xc[3 * j + k] >= o[k]) c |= (1 << k);
            oct[q] = c;
            cnt[c]++;
        }
        long start[8];
        long acc = 0;
        for (int c = 0; c < 8; ++c) { start[c] = acc; acc += cnt[c]; }
        long fill[8];
        memcpy(fill, start, sizeof(fill));
        for (long q = 0; q < n; ++q) part[fill[oct[q]]++] = idx[q];
        free(oct);
        for (int c = 0; c < 8; ++c) {
            if (cnt[c] == 0) continue;
            double lo[3], hi[3];
            long cc[3];
            for (int k = 0; k < 3; ++k) {
                int bit = (c >> k) & 1;
                lo[k] = bit ? o[k] : bmin[k];
                hi[k] = bit ? bmax[k] : o[k];
                if (!(bmax[k] > bmin[k])) { lo[k] = bmin[k]; hi[k] = bmax[k]; }
                cc[k] = 2 * cell[k] + bit;
            }
            long* sub = (long*)malloc((size_t)cnt[c] * sizeof(long));
            memcpy(sub, part + start[c], (size_t)cnt[c] * sizeof(long));
            nd->child[nd->nchild++] = create_child(T, sub, cnt[c], lo, hi, depth + 1, cc);
        }
        free(part);
        free(idx);
        nd->idx = NULL;
    } else {
        nd->idx = idx; /* leaf: a single point, or the depth limit reached */
    }
    return nd;
}

void* orc_tree_build(const double* X, const double* mX, long N, int max_depth) {
    if (N <= 0) return NULL;
    otree* T = (otree*)calloc(1, sizeof(otree));
    T->N = N;
    T->max_depth = max_depth;
    T->Xc = (double*)malloc((size_t)N * 3 * sizeof(double));
    T->m = (double*)malloc((size_t)N * sizeof(double));
    memcpy(T->Xc, X, (size_t)N * 3 * sizeof(double));
    memcpy(T->m, mX, (size_t)N * sizeof(double));
    double lo[3], hi[3];
    for (int k = 0; k < 3; ++k) { lo[k] = INFINITY; hi[k] = -INFINITY; }
    for (long j = 0; j < N; ++j)
        for (int k = 0; k < 3; ++k) {
            if (X[3 * j + k] < lo[k]) lo[k] = X[3 * j + k];
            if (X[3 * j + k] > hi[k]) hi[k] = X[3 * j + k];
        }
    long* idx = (long*)malloc((size_t)N * sizeof(long));
    for (long j = 0; j < N; ++j) idx[j] = j;
    long c0[3] = {0, 0, 0};
    T->root = create_child(T, idx, N, lo, hi, 0, c0);
    return T;
}

static void free_node(onode* nd) {
    for (int c = 0; c < nd->nchild; ++c) free_node(nd->child[c]);
    free(nd->idx);
    free(nd);
}

void orc_tree_free(void* t) {
    otree* T = (otree*)t;
    if (!T) return;
    free_node(T->root);
    free(T->Xc);
    free(T->m);
    free(T);
}

/* Canonical export. A cell with exactly one non-empty child has the same mass,
 * CoM and point set as that child; BHForce gives the same result whether such
 * a pass-through cell is visited or skipped (its l is larger, so accepting it
 * implies accepting the child). The export therefore lists only cells with
 * >= 2 children and leaves, each parent before its children (pre-order).
 * ints  per node: depth, cell x, cell y, cell z, n points, is_leaf, parent (export index or -1)
 * dbls per node: mass, com x, com y, com z, l
 * leaf_of[j]   : export index of the leaf that holds point j. */
typedef struct {
    long cap, n;
    long* ints;
    double* dbls;
    long* leaf_of;
} exporter;

static void export_rec(exporter* E, const onode* nd, long parent) {
    const onode* v = nd;
    while (v->nchild == 1) v = v->child[0]; /* skip pass-through cells */
    long me = E->n++;
    if (me < E->cap) {
        long* I = E->ints + 7 * me;
        double* D = E->dbls + 5 * me;
        I[0] = v->depth;
        I[1] = v->cell[0];
        I[2] = v->cell[1];
        I[3] = v->cell[2];
        I[4] = v->n;
        I[5] = v->nchild == 0;
        I[6] = parent;
        D[0] = v->mass;
        D[1] = v->com[0];
        D[2] = v->com[1];
        D[3] = v->com[2];
        D[4] = v->l;
        if (v->nchild == 0 && E->leaf_of)
            for (long q = 0; q < v->n; ++q) E->leaf_of[v->idx[q]] = me;
    }
    for (int c = 0; c < v->nchild; ++c) export_rec(E, v->child[c], me);
}

/* Returns the number of exported nodes (call with cap = 0 to size buffers). */
long orc_tree_export(void* t, long cap, long* ints, double* dbls, long* leaf_of) {
    otree* T = (otree*)t;
    exporter E = {cap, 0, ints, dbls, leaf_of};
    export_rec(&E, T->root, -1);
    return E.n;
}

/* Literal node count (including pass-through cells) and maximum depth. */
static void stats_rec(const onode* nd, long* count, int* maxd) {
    (*count)++;
    if (nd->depth > *maxd) *maxd = nd->depth;
    for (int c = 0; c < nd->nchild; ++c) stats_rec(nd->child[c], count, maxd);
}

void orc_tree_stats(void* t, long* literal_nodes, int* max_depth_seen) {
    otree* T = (otree*)t;
    *literal_nodes = 0;
    *max_depth_seen = 0;
    stats_rec(T->root, literal_nodes, max_depth_seen);
}

/* ------------------------------------------------------------------------ */
/* BHForce (Algorithm 2) with the opening criterion of Eq. 15                */
/* ------------------------------------------------------------------------ */

/* One monopole / particle term of Eq. 6 (without G): m (p - y) / (|p-y|^2+eps^2)^(3/2). */
static inline void add_term(const double p[3], double m, const double y[3], double e2,
                            double acc[3]) {
    double dx = p[0] - y[0], dy = p[1] - y[1], dz = p[2] - y[2];
    double w = m / pow(dx * dx + dy * dy + dz * dz + e2, 1.5);
    acc[0] += w * dx;
    acc[1] += w * dy;
    acc[2] += w * dz;
}

/* A non-empty cell whose size-to-distance ratio l / |y - CoM| is below theta
 * acts as one particle of the cell's mass at its CoM (Eq. 15). Otherwise its
 * children are visited. Reading: a leaf that fails the criterion contributes
 * each of its particles exactly (the printed recursion would drop them), the
 * recursion returns a fresh sum that the caller adds once, and a query at
 * distance 0 from the CoM fails the criterion (l / 0 is not below theta). */
static void bh_visit(const otree* T, const onode* nd, const double y[3], double theta, double e2,
                     double acc[3], long* count) {
    if (nd->n == 0) return;
    double dx = nd->com[0] - y[0], dy = nd->com[1] - y[1], dz = nd->com[2] - y[2];
    double r = sqrt(dx * dx + dy * dy + dz * dz);
    if (r > 0 && nd->l / r < theta) {
        add_term(nd->com, nd->mass, y, e2, acc);
        (*count)++;
        return;
    }
    if (nd->nchild == 0) {
        for (long q = 0; q < nd->n; ++q) {
            long j = nd->idx[q];
            add_term(T->Xc + 3 * j, T->m[j], y, e2, acc);
            (*count)++;
        }
        return;
    }
    for (int c = 0; c < nd->nchild; ++c) {
        double sub[3] = {0, 0, 0};
        bh_visit(T, nd->child[c], y, theta, e2, sub, count);
        acc[0] += sub[0];
        acc[1] += sub[1];
        acc[2] += sub[2];
    }
}

/* acc[i] = G * BHForce(root, Y_i) / m_Yi ; counts[i] = number of monopole and
 * particle terms evaluated for query i (optional). */
void orc_bh_acc(void* t, const double* Y, long M, double G, double eps, double theta, double* acc,
                long* counts) {
    otree* T = (otree*)t;
    double e2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 64)
    for (long i = 0; i < M; ++i) {
        double a[3] = {0, 0, 0};
        long c = 0;
        bh_visit(T, T->root, Y + 3 * i, theta, e2, a, &c);
        acc[3 * i] = G * a[0];
        acc[3 * i + 1] = G * a[1];
        acc[3 * i + 2] = G * a[2];
        if (counts) counts[i] = c;
    }
}

/* ------------------------------------------------------------------------ */
/* Eqs. 7-10: dissipative force, velocity and displacement                   */
/* ------------------------------------------------------------------------ */

/* f = F + F^d with F^d = -eta v (Eqs. 7-8); v' = v + dt f / m_Y (Eq. 9) where
 * F / m_Y is the gravity acceleration `acc`; d = dt v' (Eq. 10). */
void orc_ode_step(const double* v, const double* acc, const double* mY, long M, double dt,
                  double eta, double* v_out, double* d_out) {
    for (long i = 0; i < M; ++i)
        for (int k = 0; k < 3; ++k) {
            double vn = v[3 * i + k] + dt * (acc[3 * i + k] - eta * v[3 * i + k] / mY[i]);
            v_out[3 * i + k] = vn;
            d_out[3 * i + k] = dt * vn;
        }
}

/* ------------------------------------------------------------------------ */
/* Sec. IV-D: rigid projection (Eqs. 14 and 16)                              */
/* ------------------------------------------------------------------------ */

/* Singular value decomposition A = U diag(s) V^T of a 3x3 matrix by one-sided
 * (Hestenes) Jacobi rotations of the columns, singular values descending.
 * A column whose singular value is zero gets a unit vector completing U. */
static void svd3(const double A[9], double U[9], double s[3], double V[9]) {
    double W[9];
    memcpy(W, A, sizeof(W));
    for (int i = 0; i < 9; ++i) V[i] = (i % 4 == 0) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                double al = 0, be = 0, ga = 0;
                for (int i = 0; i < 3; ++i) {
                    al += W[3 * i + p] * W[3 * i + p];
                    be += W[3 * i + q] * W[3 * i + q];
                    ga += W[3 * i + p] * W[3 * i + q];
                }
                if (ga == 0.0 || fabs(ga) <= 1e-300) continue;
                double rel = fabs(ga) / sqrt(al * be);
                if (rel > off) off = rel;
                if (rel < 1e-17) continue;
                double zeta = (be - al) / (2.0 * ga);
                double tt = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + tt * tt), sn = c * tt;
                for (int i = 0; i < 3; ++i) {
                    double wp = W[3 * i + p], wq = W[3 * i + q];
                    W[3 * i + p] = c * wp - sn * wq;
                    W[3 * i + q] = sn * wp + c * wq;
                    double vp = V[3 * i + p], vq = V[3 * i + q];
                    V[3 * i + p] = c * vp - sn * vq;
                    V[3 * i + q] = sn * vp + c * vq;
                }
            }
        if (off < 1e-16) break;
    }
    double sv[3];
    for (int j = 0; j < 3; ++j)
        sv[j] = sqrt(W[j] * W[j] + W[3 + j] * W[3 + j] + W[6 + j] * W[6 + j]);
    int ord[3] = {0, 1, 2};
    for (int a = 0; a < 3; ++a)
        for (int b = a + 1; b < 3; ++b)
            if (sv[ord[b]] > sv[ord[a]]) { int tmp = ord[a]; ord[a] = ord[b]; ord[b] = tmp; }
    double Vs[9];
    memcpy(Vs, V, sizeof(Vs));
    for (int j = 0; j < 3; ++j) {
        int o = ord[j];
        s[j] = sv[o];
        for (int i = 0; i < 3; ++i) {
            V[3 * i + j] = Vs[3 * i + o];
            U[3 * i + j] = (sv[o] > 0) ? W[3 * i + o] / sv[o] : 0.0;
        }
    }
    /* complete U where a singular value vanished */
    if (!(s[2] > 0) || !(s[2] > 1e-300)) {
        double u0[3] = {U[0], U[3], U[6]}, u1[3] = {U[1], U[4], U[7]};
        U[2] = u0[1] * u1[2] - u0[2] * u1[1];
        U[5] = u0[2] * u1[0] - u0[0] * u1[2];
        U[8] = u0[0] * u1[1] - u0[1] * u1[0];
    }
}

static double det3(const double A[9]) {
    return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
           A[2] * (A[3] * A[7] - A[4] * A[6]);
}

/* Given template points Y and displacements D (both M x 3): mu_Y, mu_YD are the
 * means of Y and Y + D; C = Y^_D^T Y^ with both sets centred (Eq. 14 text);
 * C = U S V^T; R = U diag(1, 1, sgn det(U V^T)) V^T (Eq. 14); t = mu_YD - R mu_Y
 * (Eq. 16). Reading: if the second singular value is not above 1e-7 of the
 * first (a collinear or nearly collinear template), no rotation is
 * determined: R = I, t = mu_YD - mu_Y, and the return value is 1 instead of
 * 0. The bound is where an FP64 eigen-decomposition of C^T C (eigenvalues
 * sigma^2) can still tell sigma_2 from rounding: sigma_2^2 / sigma_1^2 =
 * 1e-14 is a few hundred units of the last place of sigma_1^2. */
/* Eq. 14 for D = 2 (clouds in the plane z = 0): the 2 x 2 cross-covariance
 * C = sum (y + d - mu_YD)(y - mu_Y)^T of the x, y components, its SVD
 * C = U S V^T by one Jacobi rotation (the textbook 2 x 2 case), and
 * R' = U diag(1, sgn det(U V^T)) V^T, embedded as diag(R', 1). The fit is
 * unique unless c11 + c22 and c21 - c12 both vanish (every rotation is then
 * equally good): R' = I, status 1. */
static int kabsch2(const double C3[9], double R[9]) {
    const double c11 = C3[0], c12 = C3[1], c21 = C3[3], c22 = C3[4];
    for (int i = 0; i < 9; ++i) R[i] = (i % 4 == 0) ? 1.0 : 0.0;
    const double fro = sqrt(c11 * c11 + c12 * c12 + c21 * c21 + c22 * c22);
    if (!(hypot(c11 + c22, c21 - c12) > 1e-12 * fro)) return 1;
    /* V: the rotation that diagonalises C^T C (columns a = C e1, b = C e2) */
    const double aa = c11 * c11 + c21 * c21, bb = c12 * c12 + c22 * c22, ab = c11 * c12 + c21 * c22;
    const double phi = 0.5 * atan2(2.0 * ab, aa - bb);
    const double cv = cos(phi), sv = sin(phi);
    double V[4] = {cv, -sv, sv, cv};
    /* C V = U S: columns u_k s_k */
    double W[4];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) W[2 * r + c] = C3[3 * r] * V[c] + C3[3 * r + 1] * V[2 + c];
    double s1 = hypot(W[0], W[2]), s2 = hypot(W[1], W[3]);
    double U[4];
    if (s1 < s2) { /* order the singular values */
        double t0 = W[0], t2 = W[2];
        W[0] = W[1]; W[2] = W[3]; W[1] = t0; W[3] = t2;
        double sw = s1; s1 = s2; s2 = sw;
        double v0 = V[0], v2 = V[2];
        V[0] = V[1]; V[2] = V[3]; V[1] = v0; V[3] = v2;
    }
    U[0] = W[0] / s1;
    U[2] = W[2] / s1;
    if (s2 > 0) {
        U[1] = W[1] / s2;
        U[3] = W[3] / s2;
    } else { /* rank 1: complete U to an orthonormal basis */
        U[1] = -U[2];
        U[3] = U[0];
    }
    const double detU = U[0] * U[3] - U[1] * U[2], detV = V[0] * V[3] - V[1] * V[2];
    const double sg = detU * detV < 0 ? -1.0 : 1.0;
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) R[3 * r + c] = U[2 * r] * V[2 * c] + sg * U[2 * r + 1] * V[2 * c + 1];
    return 0;
}

int orc_kabsch_d(const double* Y, const double* D, long M, int dim, double R[9], double t[3]);

int orc_kabsch(const double* Y, const double* D, long M, double R[9], double t[3]) {
    return orc_kabsch_d(Y, D, M, 3, R, t);
}

int orc_kabsch_d(const double* Y, const double* D, long M, int dim, double R[9], double t[3]) {
    double my[3] = {0, 0, 0}, myd[3] = {0, 0, 0};
    for (long i = 0; i < M; ++i)
        for (int k = 0; k < 3; ++k) {
            my[k] += Y[3 * i + k];
            myd[k] += Y[3 * i + k] + D[3 * i + k];
        }
    for (int k = 0; k < 3; ++k) { my[k] /= (double)M; myd[k] /= (double)M; }
    double C[9] = {0};
    for (long i = 0; i < M; ++i)
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                C[3 * r + c] += (Y[3 * i + r] + D[3 * i + r] - myd[r]) * (Y[3 * i + c] - my[c]);
    double U[9], s[3], V[9];
    int status = 0;
    if (dim == 2) {
        status = kabsch2(C, R);
    } else {
        svd3(C, U, s, V);
    }
    if (dim == 2) {
        /* R set by kabsch2 */
    } else if (!(s[1] > 1e-7 * s[0])) {
        for (int i = 0; i < 9; ++i) R[i] = (i % 4 == 0) ? 1.0 : 0.0;
        status = 1;
    } else {
        double UVt[9];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double acc = 0;
                for (int k = 0; k < 3; ++k) acc += U[3 * r + k] * V[3 * c + k];
                UVt[3 * r + c] = acc;
            }
        double sg = det3(UVt) < 0 ? -1.0 : 1.0;
        double Sg[3] = {1.0, 1.0, sg};
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double acc = 0;
                for (int k = 0; k < 3; ++k) acc += U[3 * r + k] * Sg[k] * V[3 * c + k];
                R[3 * r + c] = acc;
            }
    }
    for (int r = 0; r < 3; ++r)
        t[r] = myd[r] - (R[3 * r] * my[0] + R[3 * r + 1] * my[1] + R[3 * r + 2] * my[2]);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2: the FGA loop                                                 */
/* ------------------------------------------------------------------------ */

/* Inputs are already normalised (Appendix) and carry their final masses.
 * Each iteration (Algorithm 2, loop body):
 *   Y = R Y0 + t                      current template state
 *   acc = Eq. 6 (direct) or BHForce   gravity acceleration per point
 *   V, D  from Eqs. 7-10
 *   (R', t') = Kabsch(Y, D)           Eqs. 14, 16
 *   R = R' R ; t = R' t + t'          composition
 *   velocity_mode 1: v_i = (R' Y_i + t' - Y_i) / dt (the rigid motion)
 * Reading of the stopping rule: iterate while |T_k - T_{k-2}|_F^2 > conv_tol,
 * T = [R | t] accumulated (the printed condition is inverted); conv_tol <= 0
 * runs exactly max_iter iterations. V0 = 0 unless given.
 * traj (optional): [R (9, row-major), t (3)] after each iteration.
 * Returns 0, or the number of iterations whose rigid fit was degenerate. */
int orc_register(const double* Xn, const double* mX, long N, const double* Yn, const double* mY,
                 long M, const orc_params* p, const double* V0, double R[9], double t[3],
                 int* iters, double* traj, long* interactions, double* V_out) {
    double* Y = (double*)malloc((size_t)M * 3 * sizeof(double));
    double* V = (double*)calloc((size_t)M * 3, sizeof(double));
    double* A = (double*)malloc((size_t)M * 3 * sizeof(double));
    double* Dd = (double*)malloc((size_t)M * 3 * sizeof(double));
    long* cnt = (long*)malloc((size_t)M * sizeof(long));
    if (V0) memcpy(V, V0, (size_t)M * 3 * sizeof(double));
    void* tree = NULL;
    if (p->method == 1) tree = orc_tree_build(Xn, mX, N, p->max_depth);
    for (int i = 0; i < 9; ++i) R[i] = (i % 4 == 0) ? 1.0 : 0.0;
    t[0] = t[1] = t[2] = 0.0;
    double hist[2][12];
    int degenerate = 0;
    long total = 0;
    int k;
    for (k = 0; k < p->max_iter; ++k) {
        for (long i = 0; i < M; ++i)
            for (int r = 0; r < 3; ++r)
                Y[3 * i + r] = R[3 * r] * Yn[3 * i] + R[3 * r + 1] * Yn[3 * i + 1] +
                               R[3 * r + 2] * Yn[3 * i + 2] + t[r];
        if (p->method == 1) {
            orc_bh_acc(tree, Y, M, p->G, p->eps, p->theta, A, cnt);
            for (long i = 0; i < M; ++i) total += cnt[i];
        } else {
            orc_direct_acc(Xn, mX, N, Y, M, p->G, p->eps, A, NULL);
            total += (long)N * M;
        }
        orc_ode_step(V, A, mY, M, p->dt, p->eta, V, Dd);
        double Rp[9], tp[3];
        degenerate += orc_kabsch_d(Y, Dd, M, p->dim == 2 ? 2 : 3, Rp, tp);
        double Rn[9], tn[3];
        for (int r = 0; r < 3; ++r) {
            for (int c = 0; c < 3; ++c)
                Rn[3 * r + c] =
                    Rp[3 * r] * R[c] + Rp[3 * r + 1] * R[3 + c] + Rp[3 * r + 2] * R[6 + c];
            tn[r] = Rp[3 * r] * t[0] + Rp[3 * r + 1] * t[1] + Rp[3 * r + 2] * t[2] + tp[r];
        }
        memcpy(R, Rn, sizeof(Rn));
        memcpy(t, tn, sizeof(tn));
        if (p->velocity_mode == 1) {
            for (long i = 0; i < M; ++i)
                for (int r = 0; r < 3; ++r) {
                    double moved = Rp[3 * r] * Y[3 * i] + Rp[3 * r + 1] * Y[3 * i + 1] +
                                   Rp[3 * r + 2] * Y[3 * i + 2] + tp[r];
                    V[3 * i + r] = (moved - Y[3 * i + r]) / p->dt;
                }
        }
        double cur[12];
        memcpy(cur, R, 9 * sizeof(double));
        memcpy(cur + 9, t, 3 * sizeof(double));
        if (traj) memcpy(traj + 12 * k, cur, sizeof(cur));
        int stop = 0;
        if (p->conv_tol > 0 && k >= 2) {
            double d2 = 0;
            for (int q = 0; q < 12; ++q) d2 += (cur[q] - hist[k % 2][q]) * (cur[q] - hist[k % 2][q]);
            if (d2 <= p->conv_tol) stop = 1;
        }
        memcpy(hist[k % 2], cur, sizeof(cur));
        if (stop) { ++k; break; }
    }
    if (iters) *iters = k;
    if (interactions) *interactions = total;
    if (V_out) memcpy(V_out, V, (size_t)M * 3 * sizeof(double));
    orc_tree_free(tree);
    free(Y);
    free(V);
    free(A);
    free(Dd);
    free(cnt);
    return degenerate;
}
