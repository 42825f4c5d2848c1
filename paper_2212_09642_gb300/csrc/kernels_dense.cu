// Small dense kernels of libvne: the tridiagonal eigensolve + Gauss
// quadrature (Section 4, eq. rational-krylov-approximation-quadform), the
// Lanczos matvec coefficients f(T) e1, and the Hutch++ sketch linear algebra
// (Gram matrices, block products, pivoted Cholesky-QR factor).
//
// Tridiagonal eigenproblems use the implicit symmetric QR iteration with a
// Wilkinson shift (Golub & Van Loan, Matrix Computations, Sec. 8.3), in
// FP64.  Only the first row of the eigenvector matrix is needed for the
// quadrature (the Golub-Welsch weights u_{1j}^2), so the per-column kernel
// tracks that row alone; the matvec kernel keeps the full eigenvector matrix
// in shared memory, one warp per column, lanes owning its rows.
#include <float.h>
#include <math.h>
#include <stdlib.h>

#include "kernels.h"

namespace vne {

__host__ __device__ __forceinline__ double f_entropy(double x) { return x > 0.0 ? -x * log(x) : 0.0; }

#ifndef __CUDA_ARCH__
static inline double rsqrt(double v) { return 1.0 / sqrt(v); }
#endif

// One implicit QR sweep framework.  d[0..n), e[0..n-1) are overwritten by the
// eigenvalues / zeros; `rot(k, c, s)` is called for every Givens rotation
// acting on columns k, k+1 of the eigenvector matrix.  Returns false if the
// iteration cap was hit.
template <typename Rot>
__host__ __device__ bool symtri_qr(double* d, double* e, int n, Rot rot) {
    const double eps = DBL_EPSILON;
    int hi = n - 1;
    int iters = 0;
    const int max_iters = 40 * n + 40;
    while (hi > 0) {
        if (fabs(e[hi - 1]) <= eps * (fabs(d[hi - 1]) + fabs(d[hi]))) {
            e[hi - 1] = 0.0;
            hi--;
            continue;
        }
        int lo = hi - 1;
        while (lo > 0 && fabs(e[lo - 1]) > eps * (fabs(d[lo - 1]) + fabs(d[lo]))) lo--;
        if (lo > 0) e[lo - 1] = 0.0;
        if (++iters > max_iters) return false;
        // Wilkinson shift: eigenvalue of the trailing 2x2 closer to d[hi]
        double delta = 0.5 * (d[hi - 1] - d[hi]);
        double b2 = e[hi - 1] * e[hi - 1];
        double den = delta + copysign(sqrt(delta * delta + b2), delta == 0.0 ? 1.0 : delta);
        double mu = d[hi] - b2 / den;
        double x = d[lo] - mu, y = e[lo];
        for (int k = lo; k < hi; k++) {
            // Givens rotation from one reciprocal square root (cheaper than
            // hypot and two divisions on an FP64-poor GPU)
            double r2 = x * x + y * y;
            double c, s, r;
            if (r2 == 0.0) {
                c = 1.0;
                s = 0.0;
                r = 0.0;
            } else {
                double inv = rsqrt(r2);
                c = x * inv;
                s = -y * inv;
                r = r2 * inv;
            }
            if (k > lo) e[k - 1] = r;
            double a = d[k], b = e[k], cc = d[k + 1];
            double cs = c * s, c2 = c * c, s2 = s * s;
            d[k] = a * c2 - 2.0 * b * cs + cc * s2;
            d[k + 1] = a * s2 + 2.0 * b * cs + cc * c2;
            e[k] = (a - cc) * cs + b * (c2 - s2);
            rot(k, c, s);
            if (k < hi - 1) {
                x = e[k];
                y = -s * e[k + 1];
                e[k + 1] = c * e[k + 1];
            }
        }
    }
    return true;
}

// Implicit QR with `nr` rows of the eigenvector matrix tracked alongside (the
// quadrature needs the first row only; f(T) e1 needs all rows, spread over
// the lanes of a warp).  The sweep's running values (d_k, e_k and each
// tracked row's entry k) are carried in registers, so the dependent chain of
// one rotation touches no memory; old values of the next position are loaded
// ahead of their use.
template <int R>
__host__ __device__ inline bool symtri_qr_rows(double* d, double* e, int n, double* const* zr, int nr) {
    const double eps = DBL_EPSILON;
    int hi = n - 1;
    int iters = 0;
    const int max_iters = 40 * n + 40;
    while (hi > 0) {
        if (fabs(e[hi - 1]) <= eps * (fabs(d[hi - 1]) + fabs(d[hi]))) {
            e[hi - 1] = 0.0;
            hi--;
            continue;
        }
        int lo = hi - 1;
        while (lo > 0 && fabs(e[lo - 1]) > eps * (fabs(d[lo - 1]) + fabs(d[lo]))) lo--;
        if (lo > 0) e[lo - 1] = 0.0;
        if (++iters > max_iters) return false;
        const double delta = 0.5 * (d[hi - 1] - d[hi]);
        const double b2 = e[hi - 1] * e[hi - 1];
        const double den = delta + copysign(sqrt(delta * delta + b2), delta == 0.0 ? 1.0 : delta);
        const double mu = d[hi] - b2 / den;
        double dk = d[lo], ek = e[lo];
        double zk[R];
#pragma unroll
        for (int q = 0; q < R; q++) zk[q] = (q < nr) ? zr[q][lo] : 0.0;
        double x = dk - mu, y = ek;
        for (int k = lo; k < hi; k++) {
            const double dk1 = d[k + 1];
            const double ek1 = (k + 1 < hi) ? e[k + 1] : 0.0;
            double zk1[R];
#pragma unroll
            for (int q = 0; q < R; q++) zk1[q] = (q < nr) ? zr[q][k + 1] : 0.0;
            const double r2 = x * x + y * y;
            double c, s, r;
            if (r2 == 0.0) {
                c = 1.0;
                s = 0.0;
                r = 0.0;
            } else {
                const double inv = rsqrt(r2);
                c = x * inv;
                s = -y * inv;
                r = r2 * inv;
            }
            if (k > lo) e[k - 1] = r;
            const double cs = c * s, c2 = c * c, s2 = s * s;
            const double a = dk, b = ek;
            d[k] = a * c2 - 2.0 * b * cs + dk1 * s2;
            const double ndk1 = a * s2 + 2.0 * b * cs + dk1 * c2;
            const double nek = (a - dk1) * cs + b * (c2 - s2);
#pragma unroll
            for (int q = 0; q < R; q++) {
                if (q < nr) zr[q][k] = c * zk[q] - s * zk1[q];
                zk[q] = s * zk[q] + c * zk1[q];
            }
            dk = ndk1;
            if (k < hi - 1) {
                x = nek;
                y = -s * ek1;
                ek = c * ek1;
            } else {
                e[k] = nek;
            }
        }
        d[hi] = dk;
#pragma unroll
        for (int q = 0; q < R; q++)
            if (q < nr) zr[q][hi] = zk[q];
    }
    return true;
}

__host__ __device__ inline bool symtri_qr_first_row(double* d, double* e, double* z, int n) {
    double* rows[1] = {z};
    return symtri_qr_rows<1>(d, e, n, rows, 1);
}

// ---------------------------------------------------------------------------
// Gauss quadrature psi = ||c||^2 sum_j u_{1j}^2 f(sigma theta_j) of the
// leading unreduced block of T (Golub & Meurant, Matrices, Moments and
// Quadrature, Ch. 6), one warp per tridiagonal with the eigenvalues spread
// over the lanes.  GB300 retires FP64 instructions slowly and with long
// latency, so one long sequential QR chain per column is the slowest possible
// schedule; here every lane runs short independent chains:
//  * theta_j by bisection on the Sturm count #{theta < z} (number of k with
//    sign p_k(z) = sign p_{k-1}(z), p_k = det(z I - T_k) by the three-term
//    recurrence, rescaled by powers of two every four steps; Wilkinson, The
//    Algebraic Eigenvalue Problem, Ch. 5): FP32 halvings first narrow the
//    Gershgorin interval, FP64 counts check the bracket, then FP64
//    quadrisection with all of a lane's points evaluated as interleaved
//    independent recurrences, a warp-uniform number of passes;
//  * u_{1j}^2 from the eigenvector of the twisted factorisation
//    T - theta I = N_r Delta_r N_r^T at the twist index r of smallest
//    |gamma_r| (Parlett & Dhillon, Lin. Alg. Appl. 309, 2000): z_r = 1,
//    components above r from the top-down pivots, below r from the bottom-up
//    pivots, u_{1j}^2 = z_1^2 / ||z||^2;
//  * eigenvalues closer than kClusterGap * span to a neighbour (or closer
//    than 16 x the half-width of the group being formed) form a cluster,
//    whose individual weights are ill-conditioned; its summed weight W and
//    first and second moments come from the resolvent e1^T (z I - T)^{-1} e1
//    (continued fraction) integrated by the trapezoid rule on a circle
//    around it, and it contributes W f(tbar) + f''(tbar) W var / 2 (weighted
//    mean tbar, variance var).  A cluster closer than 16 x its half-width to
//    the previous group sends the column to the sequential implicit QR
//    (lane 0), which keeps the kernel correct for any input.
constexpr double kClusterGap = 1e-5;
constexpr int kContourPoints = 32;

// Power of two that brings |x| (the largest of the values passed) to [1, 2):
// multiplying the recurrence state by it keeps signs and ratios.
__device__ __forceinline__ double pow2_rescale(long long maxbits) {
    int se = 2046 - (int)(maxbits >> 52);
    se = se < 1 ? 1 : (se > 2046 ? 2046 : se);
    return __longlong_as_double((long long)se << 52);
}

__device__ __forceinline__ long long absbits(double x) { return __double_as_longlong(x) & 0x7fffffffffffffffLL; }

// #{eigenvalues of the leading n x n block < z[q]} for NC points at once
// (independent recurrences, interleaved for instruction-level parallelism):
// the number of k with sign p_k = sign p_{k-1}, p_0 = 1.  b2[k] =
// beta_{k-1}^2, b2[0] = 0.  A p_k that is exactly +0 counts as positive (a
// perturbation of z by one ulp).
template <int NC>
__device__ __forceinline__ void sturm_counts(const double* a, const double* b2, int n, const double (&z)[NC],
                                             int (&cnt)[NC]) {
    double p2[NC], p1[NC];  // p_{k-2}, p_{k-1}
    int hprev[NC], changes[NC];
#pragma unroll
    for (int q = 0; q < NC; q++) {
        p2[q] = 0.0;
        p1[q] = 1.0;
        hprev[q] = 0;
        changes[q] = 0;
    }
    for (int k = 0; k < n; k++) {
        const double ak = a[k], bk = b2[k];
#pragma unroll
        for (int q = 0; q < NC; q++) {
            const double p = fma(z[q] - ak, p1[q], -(bk * p2[q]));
            const int h = __double2hiint(p);
            changes[q] += (int)((unsigned)(h ^ hprev[q]) >> 31);
            hprev[q] = h;
            p2[q] = p1[q];
            p1[q] = p;
        }
        if ((k & 7) == 7) {
#pragma unroll
            for (int q = 0; q < NC; q++) {
                const long long m1 = absbits(p1[q]), m2 = absbits(p2[q]);
                const double fsc = pow2_rescale(m1 > m2 ? m1 : m2);
                p1[q] *= fsc;
                p2[q] *= fsc;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < NC; q++) cnt[q] = n - changes[q];
}

// p_n(z) / p_n'(z) for the characteristic polynomial p_n(z) = det(z I - T)
// and the Sturm count at z, from one recurrence (p_k' = p_{k-1} +
// (z - a_k) p_{k-1}' - b2_k p_{k-2}'), for NC points.
template <int NC>
__device__ __forceinline__ void newton_counts(const double* a, const double* b2, int n, const double (&z)[NC],
                                              double (&ratio)[NC], int (&cnt)[NC]) {
    double p2[NC], p1[NC], d2[NC], d1[NC];
    int hprev[NC], changes[NC];
#pragma unroll
    for (int q = 0; q < NC; q++) {
        p2[q] = 0.0;
        p1[q] = 1.0;
        d2[q] = 0.0;
        d1[q] = 0.0;
        hprev[q] = 0;
        changes[q] = 0;
    }
    for (int k = 0; k < n; k++) {
        const double ak = a[k], bk = b2[k];
#pragma unroll
        for (int q = 0; q < NC; q++) {
            const double zk = z[q] - ak;
            const double p = fma(zk, p1[q], -(bk * p2[q]));
            const double d = fma(zk, d1[q], p1[q]) - bk * d2[q];
            const int h = __double2hiint(p);
            changes[q] += (int)((unsigned)(h ^ hprev[q]) >> 31);
            hprev[q] = h;
            p2[q] = p1[q];
            p1[q] = p;
            d2[q] = d1[q];
            d1[q] = d;
        }
        if ((k & 7) == 7) {
#pragma unroll
            for (int q = 0; q < NC; q++) {
                long long m = absbits(p1[q]);
                m = max(m, absbits(p2[q]));
                m = max(m, absbits(d1[q]));
                m = max(m, absbits(d2[q]));
                const double fsc = pow2_rescale(m);
                p1[q] *= fsc;
                p2[q] *= fsc;
                d1[q] *= fsc;
                d2[q] *= fsc;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < NC; q++) {
        ratio[q] = p1[q] / d1[q];
        cnt[q] = n - changes[q];
    }
}

// FP32 Sturm count on the FP32-rounded block (pivots d_k of T - zI,
// #{d_k < 0}), used only to narrow the FP64 search interval; the interval is
// checked with FP64 counts before it is trusted.
__device__ __forceinline__ int sturm_count_f32(const float* a, const float* b2, int n, float z, float pivmin) {
    int cnt = 0;
    float d = 1.f;
    for (int k = 0; k < n; k++) {
        d = (a[k] - z) - __fdividef(b2[k], d);
        if (fabsf(d) < pivmin) d = -pivmin;
        cnt += d < 0.f;
    }
    return cnt;
}

__device__ __forceinline__ double guard_pivot(double x, double pivmin) {
    return fabs(x) < pivmin ? (x < 0.0 ? -pivmin : pivmin) : x;
}

// u_{1j}^2 by the twisted factorisation at an isolated eigenvalue th.
// Dp / Rp: this lane's columns of the pivot scratch ([k][32] doubles).
__device__ double twisted_weight(const double* a, const double* b, int n, double th, double pivmin, double* Dp,
                                 double* Rp) {
    double d = 0.0;
    for (int k = 0; k < n; k++) {
        d = guard_pivot((a[k] - th) - (k > 0 ? b[k - 1] * b[k - 1] / d : 0.0), pivmin);
        Dp[k * 32] = d;
    }
    double r = 0.0, best = INFINITY;
    int tw = n - 1;
    for (int k = n - 1; k >= 0; k--) {
        r = guard_pivot((a[k] - th) - (k + 1 < n ? b[k] * b[k] / r : 0.0), pivmin);
        Rp[k * 32] = r;
        const double gam = fabs(Dp[k * 32] + r - (a[k] - th));
        if (gam < best) {
            best = gam;
            tw = k;
        }
    }
    double s = 1.0, z = 1.0;
    for (int k = tw - 1; k >= 0; k--) {
        z = -b[k] * z / Dp[k * 32];
        s = fma(z, z, s);
    }
    const double z1 = tw > 0 ? z : 1.0;
    z = 1.0;
    for (int k = tw + 1; k < n; k++) {
        z = -b[k - 1] * z / Rp[k * 32];
        s = fma(z, z, s);
    }
    return z1 * z1 / s;
}

// Point q of the K-point trapezoid rule on the circle z = c + rho e^{i phi}:
// Re F(z) dz^p, p = 1, 2, 3, with dz = z - c and F(z) = e1^T (z I - T)^{-1} e1
// by the bottom-up continued fraction.  (1/K) times their sums over q are the
// summed weight and the first and second moments about c of the eigenvalues
// inside the circle.
__device__ void resolvent_point(const double* a, const double* b, int n, double c, double rho, int q, double& re1,
                                double& re2, double& re3) {
    double sph, cph;
    sincospi((2.0 * q + 1.0) / kContourPoints, &sph, &cph);
    const double dzr = rho * cph, dzi = rho * sph;
    const double zr = c + dzr, zi = dzi;
    double gr = zr - a[n - 1], gi = zi;
    for (int k = n - 2; k >= 0; k--) {
        // g <- (z - a_k) - b_k^2 / g
        const double t = b[k] * b[k] / (gr * gr + gi * gi);
        gr = (zr - a[k]) - t * gr;
        gi = zi + t * gi;
    }
    const double den = gr * gr + gi * gi;
    const double fr = gr / den, fi = -gi / den;                        // F = 1 / g
    const double pr = fr * dzr - fi * dzi, pim = fr * dzi + fi * dzr;  // F dz
    re1 = pr;
    const double p2r = pr * dzr - pim * dzi, p2i = pr * dzi + pim * dzr;  // F dz^2
    re2 = p2r;
    re3 = p2r * dzr - p2i * dzi;  // Re(F dz^3)
}

// Fallback: the quadrature by the sequential implicit QR of the whole
// (scaled) block, run by lane 0 of the warp.
template <int MAXM>
__device__ void quad_by_qr(const double* sa, const double* sb, int n, double sc, double norm2, int lane,
                           double* out) {
    if (lane != 0) return;
    double d[MAXM], ee[MAXM], z[MAXM];
    for (int k = 0; k < n; k++) {
        d[k] = sa[k];
        ee[k] = sb[k];
        z[k] = 0.0;
    }
    z[0] = 1.0;
    const bool ok = symtri_qr_first_row(d, ee, z, n);
    double s = 0.0;
    for (int k = 0; k < n; k++) s += z[k] * z[k] * f_entropy(sc * d[k]);
    *out = ok ? norm2 * s : nan("");
}

// Shared state of the spectral kernels for one tridiagonal (one warp).
template <int MAXM>
struct TqShared {
    double a[MAXM], b[MAXM], b2[MAXM + 1];  // scaled block, b2[k] = beta_{k-1}^2
    double th[MAXM], bw[MAXM];              // eigenvalues (ascending), bracket widths
    float a32[MAXM], b2_32[MAXM + 1];
    double cc[MAXM / 2], rho[MAXM / 2], half[MAXM / 2];  // clusters: centre, circle radius, half-width
    int gfirst[MAXM + 1], glast[MAXM], cl_of_group[MAXM];
    int ngroups, ncl, fallback, n;
    double span, s2, pivmin;
};

// Eigenvalues and their grouping for the leading unreduced block of
// tridiagonal c (all 32 lanes call it).  Returns false if the block has a
// non-finite entry.
template <int MAXM>
__device__ bool tq_spectrum(const double* __restrict__ alpha, const double* __restrict__ beta, int c, int m, int ld,
                            int lane, TqShared<MAXM>& S) {
    double* sa = S.a;
    double* sb = S.b;
    double* sb2 = S.b2;
    double* sth = S.th;
    double* sbw = S.bw;
    float* sa32 = S.a32;
    float* sb2_32 = S.b2_32;
    // leading unreduced block: n = 1 + first j with beta_j == 0
    int n = m;
    for (int j0 = 0; j0 < m - 1; j0 += 32) {
        const int j = j0 + lane;
        const bool zero = j < m - 1 && beta[(size_t)j * ld + c] == 0.0;
        const unsigned zb = __ballot_sync(0xffffffffu, zero);
        if (zb) {
            n = j0 + __ffs(zb);
            break;
        }
    }
    bool finite = true;
    double glo = INFINITY, ghi = -INFINITY, bmax = 0.0;
    for (int j = lane; j < n; j += 32) {
        const double aj = alpha[(size_t)j * ld + c];
        const double bj = (j + 1 < n) ? beta[(size_t)j * ld + c] : 0.0;
        const double bp = (j > 0) ? beta[(size_t)(j - 1) * ld + c] : 0.0;
        sa[j] = aj;
        sb[j] = bj;
        sb2[j + 1] = bj * bj;
        finite = finite && isfinite(aj) && isfinite(bj);
        const double r = fabs(bj) + fabs(bp);
        glo = fmin(glo, aj - r);
        ghi = fmax(ghi, aj + r);
        bmax = fmax(bmax, bj * bj);
    }
    if (lane == 0) {
        sb2[0] = 0.0;
        sb2_32[0] = 0.f;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        glo = fmin(glo, __shfl_xor_sync(0xffffffffu, glo, off));
        ghi = fmax(ghi, __shfl_xor_sync(0xffffffffu, ghi, off));
        bmax = fmax(bmax, __shfl_xor_sync(0xffffffffu, bmax, off));
    }
    finite = __all_sync(0xffffffffu, finite);
    __syncwarp();
    if (!finite) return false;
    // scale the block by the power of two s2 that brings its Gershgorin
    // radius to [1, 2) (exact: eigenvalues scale by s2, weights do not), so
    // the unnormalised Sturm recurrences stay far from overflow
    const double s2 = pow2_rescale(absbits(fmax(fmax(fabs(glo), fabs(ghi)), DBL_MIN)));
    for (int j = lane; j < n; j += 32) {
        sa[j] *= s2;
        sb[j] *= s2;
        sb2[j + 1] *= s2 * s2;
        sa32[j] = (float)sa[j];
        sb2_32[j + 1] = (float)sb2[j + 1];
    }
    __syncwarp();
    glo *= s2;
    ghi *= s2;
    bmax *= s2 * s2;
    const double span = fmax(fmax(fabs(glo), fabs(ghi)), DBL_MIN);
    glo -= 4.0 * DBL_EPSILON * span + DBL_MIN;
    ghi += 4.0 * DBL_EPSILON * span + DBL_MIN;
    const double pivmin = DBL_MIN * fmax(1.0, bmax);
    // 1. eigenvalues, ascending: theta_j is the j-th smallest.  Lane l owns
    //    j = l + 32 r, r < R (the last lanes carry a dummy root when n < 32 R,
    //    so the warp stays converged).
    constexpr int R = MAXM / 32;
    double lo[R], hi[R];
    int clo[R], chi[R];  // Sturm counts at lo and hi
    {
        // (a) FP32 bisection narrows each bracket to a few ulps of FP32
        const float pivmin32 = FLT_MIN * fmaxf(1.f, (float)bmax);
        const float glo32 = (float)glo, ghi32 = (float)ghi;
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int j = lane + 32 * r;
            float l32 = glo32, h32 = ghi32;
            if (j < n)
                for (int it = 0; it < 26; it++) {
                    const float z = 0.5f * (l32 + h32);
                    if (sturm_count_f32(sa32, sb2_32, n, z, pivmin32) > j) h32 = z;
                    else l32 = z;
                }
            const double w = 4e-6 * span + 8.0 * (double)FLT_EPSILON * fabs((double)h32);
            lo[r] = fmax(glo, (double)l32 - w);
            hi[r] = fmin(ghi, (double)h32 + w);
        }
        // (b) FP64 check of the brackets: count(lo) <= j < count(hi)
        double zc[2 * R];
        int cc[2 * R];
#pragma unroll
        for (int r = 0; r < R; r++) {
            zc[2 * r] = lo[r];
            zc[2 * r + 1] = hi[r];
        }
        sturm_counts<2 * R>(sa, sb2, n, zc, cc);
        bool widened = false;
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int j = lane + 32 * r;
            clo[r] = cc[2 * r];
            chi[r] = cc[2 * r + 1];
            if (j < n && !(clo[r] <= j && chi[r] > j)) {
                lo[r] = glo;
                hi[r] = ghi;
                clo[r] = 0;
                chi[r] = n;
                widened = true;
            }
        }
        // (c) FP64 quadrisection (three interior points per root and pass)
        //     down to ~3e-8 span: 4 passes from the FP32 bracket, 13 from the
        //     Gershgorin interval
        const int passes = __any_sync(0xffffffffu, widened) ? 13 : 4;
        for (int it = 0; it < passes; it++) {
            double zq[3 * R];
            int cq[3 * R];
#pragma unroll
            for (int r = 0; r < R; r++) {
                const double w = hi[r] - lo[r];
#pragma unroll
                for (int q = 0; q < 3; q++) zq[3 * r + q] = lo[r] + 0.25 * (q + 1) * w;
            }
            sturm_counts<3 * R>(sa, sb2, n, zq, cq);
#pragma unroll
            for (int r = 0; r < R; r++) {
                const int j = lane + 32 * r;
                const double z1 = zq[3 * r], z2 = zq[3 * r + 1], z3 = zq[3 * r + 2];
                if (cq[3 * r] > j) {
                    hi[r] = z1;
                    chi[r] = cq[3 * r];
                } else if (cq[3 * r + 1] > j) {
                    lo[r] = z1;
                    clo[r] = cq[3 * r];
                    hi[r] = z2;
                    chi[r] = cq[3 * r + 1];
                } else if (cq[3 * r + 2] > j) {
                    lo[r] = z2;
                    clo[r] = cq[3 * r + 1];
                    hi[r] = z3;
                    chi[r] = cq[3 * r + 2];
                } else {
                    lo[r] = z3;
                    clo[r] = cq[3 * r + 2];
                }
            }
        }
        // (d) safeguarded Newton on p_n (each step also counts, so the bracket
        //     keeps shrinking): a root alone in its bracket converges
        //     quadratically; roots sharing a bracket (tight clusters) keep
        //     the bracket midpoint and are handled as a cluster below
        double zn[R];
#pragma unroll
        for (int r = 0; r < R; r++) zn[r] = 0.5 * (lo[r] + hi[r]);
        for (int it = 0; it < 4; it++) {
            double ratio[R];
            int cn[R];
            newton_counts<R>(sa, sb2, n, zn, ratio, cn);
#pragma unroll
            for (int r = 0; r < R; r++) {
                const int j = lane + 32 * r;
                if (cn[r] > j) {
                    hi[r] = zn[r];
                    chi[r] = cn[r];
                } else {
                    lo[r] = zn[r];
                    clo[r] = cn[r];
                }
                const double zt = zn[r] - ratio[r];
                const bool alone = (chi[r] - clo[r]) == 1;
                zn[r] = (alone && zt >= lo[r] && zt <= hi[r]) ? zt : 0.5 * (lo[r] + hi[r]);  // converged: stays
            }
        }
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int j = lane + 32 * r;
            if (j < n) {
                sth[j] = zn[r];
                sbw[j] = hi[r] - lo[r];
            }
        }
    }
    __syncwarp();
    // 2. groups of eigenvalues (lane 0, one pass with merging): a group grows
    //    while the next gap is below kClusterGap * span or below 16 x its
    //    half-width, and absorbs the previous group while the gap to it is
    //    below 17 x its half-width; one-member groups are isolated
    //    eigenvalues, the others clusters.  A cluster closer than 16 x its
    //    half-width to a neighbouring group sends the column to the
    //    sequential QR.
    const double tau = kClusterGap * span;
    double* s_cc = S.cc;
    double* s_rho = S.rho;
    double* s_half = S.half;
    int* s_gfirst = S.gfirst;
    int* s_glast = S.glast;
    int* s_cl_of_group = S.cl_of_group;
    if (lane == 0) {
        auto halfw = [&](int f, int l) {
            double h = 0.5 * (sth[l] - sth[f]);
            for (int q = f; q <= l; q++) h = fmax(h, 0.5 * sbw[q]);
            return h;
        };
        int ng = 0;
        for (int j = 0; j < n;) {
            int f = j, e = j;
            for (;;) {
                while (e + 1 < n) {
                    const double gap = sth[e + 1] - sth[e];
                    if (!(gap < tau || gap < 16.0 * halfw(f, e))) break;
                    e++;
                }
                if (ng > 0 && e > f && sth[f] - sth[s_glast[ng - 1]] < 17.0 * halfw(f, e)) {
                    f = s_gfirst[--ng];  // absorb the previous group
                    continue;
                }
                break;
            }
            s_gfirst[ng] = f;
            s_glast[ng] = e;
            ng++;
            j = e + 1;
        }
        int ncl = 0, fb = 0;
        for (int g = 0; g < ng; g++) {
            const int f = s_gfirst[g], e = s_glast[g];
            s_cl_of_group[g] = -1;
            if (e == f) continue;
            const double half = fmax(halfw(f, e), 4.0 * DBL_EPSILON * span);
            const double dl = g > 0 ? sth[f] - sth[s_glast[g - 1]] : INFINITY;
            const double dr = g + 1 < ng ? sth[s_gfirst[g + 1]] - sth[e] : INFINITY;
            const double D = fmin(dl, dr) - half;
            if (!(D >= 16.0 * half)) fb = 1;
            // circle radius: D / 8 for a tight cluster, else the geometric mean
            // of half-width and distance (both error terms (half / D)^(K/2))
            s_cc[ncl] = 0.5 * (sth[f] + sth[e]);
            s_rho[ncl] = !isfinite(D) ? 0.25 * span : (D >= 64.0 * half ? D / 8.0 : sqrt(half * D));
            s_half[ncl] = half;
            s_cl_of_group[g] = ncl++;
        }
        s_gfirst[ng] = n;
        S.ngroups = ng;
        S.ncl = ncl;
        S.fallback = fb;
        S.n = n;
        S.span = span;
        S.s2 = s2;
        S.pivmin = pivmin;
    }
    __syncwarp();
    return true;
}

template <int MAXM>
__global__ void __launch_bounds__(32) k_tridiag_quad(const double* __restrict__ alpha, const double* __restrict__ beta,
                                                     const double* __restrict__ norm2, const double* __restrict__ scale,
                                                     int count, int m_all, int ld, double* __restrict__ psi,
                                                     const int32_t* __restrict__ cols,
                                                     const int32_t* __restrict__ mcol) {
    __shared__ TqShared<MAXM> S;
    extern __shared__ double piv[];  // [2][MAXM][32]: twisted pivots, transposed per lane
    const int lane = threadIdx.x;
    if ((int)blockIdx.x >= count) return;
    // entry blockIdx.x: column c (of the ld-strided arrays) after m steps
    const int c = cols ? cols[blockIdx.x] : (int)blockIdx.x;
    const int m = mcol ? mcol[blockIdx.x] : m_all;
    if (!tq_spectrum<MAXM>(alpha, beta, c, m, ld, lane, S)) {
        if (lane == 0) psi[c] = nan("");
        return;
    }
    const int n = S.n;
    const double span = S.span, pivmin = S.pivmin;
    const double* sa = S.a;
    const double* sb = S.b;
    const double* sth = S.th;
    const double* s_cc = S.cc;
    const double* s_rho = S.rho;
    const double* s_half = S.half;
    const int* s_gfirst = S.gfirst;
    const int* s_cl_of_group = S.cl_of_group;
    const double sc = scale[c] / S.s2;  // f is applied to the unscaled eigenvalues
    const int ngroups = S.ngroups, ncl = S.ncl;
    if (S.fallback) {
        quad_by_qr<MAXM>(sa, sb, n, sc, norm2[c], lane, psi + c);
        return;
    }
    // 3. isolated eigenvalues: twisted-factorisation weights, groups spread
    //    over the lanes
    double acc = 0.0, wsum = 0.0, errb = 0.0;
    for (int g = lane; g < ngroups; g += 32) {
        if (s_cl_of_group[g] >= 0) continue;
        const int j = s_gfirst[g];
        const double w = twisted_weight(sa, sb, n, sth[j], pivmin, piv + lane, piv + MAXM * 32 + lane);
        acc += w * f_entropy(sc * sth[j]);
        wsum += w;
    }
    // 4. clusters: the K contour points of all clusters spread over the lanes
    //    (their values reuse the pivot scratch), then lane (cluster mod 32)
    //    sums each cluster's points in order
    __syncwarp();
    double* pts = piv;  // [cluster][K][3]
    for (int item = lane; item < ncl * kContourPoints; item += 32) {
        const int cl = item / kContourPoints, q = item % kContourPoints;
        resolvent_point(sa, sb, n, s_cc[cl], s_rho[cl], q, pts[3 * item], pts[3 * item + 1], pts[3 * item + 2]);
    }
    __syncwarp();
    for (int cl = lane; cl < ncl; cl += 32) {
        double W = 0.0, M1 = 0.0, M2 = 0.0;
        for (int q = 0; q < kContourPoints; q++) {
            W += pts[3 * (cl * kContourPoints + q)];
            M1 += pts[3 * (cl * kContourPoints + q) + 1];
            M2 += pts[3 * (cl * kContourPoints + q) + 2];
        }
        W /= kContourPoints;
        M1 /= kContourPoints;
        M2 /= kContourPoints;
        // sum_j w_j f(theta_j) over the cluster ~ W f(tbar) + f''(tbar) W var / 2
        // with the weighted mean tbar and variance var; a cluster whose weight
        // is at rounding level (eigenvectors that vanish at row 1) keeps its
        // centre and no correction
        const double cc = s_cc[cl], half = s_half[cl];
        double contrib = W * f_entropy(sc * cc);
        if (W > 0.0 && fabs(M1) <= 2.0 * half * W) {
            const double mu = M1 / W, tbar = cc + mu;
            const double var = fmax(M2 / W - mu * mu, 0.0);
            contrib = W * f_entropy(sc * tbar);
            if (tbar > 0.0) contrib -= 0.5 * (sc / tbar) * W * var;  // d2/dt2 f(sc t) = -sc / t
        }
        if (half > 1e-3 * fabs(cc)) {
            // a cluster at the origin: the expansion does not hold, but its
            // members lie in [cc - half, cc + half] and f >= 0 increases from
            // 0, so the error is below W f(cc + half)
            errb += fmax(W, 0.0) * f_entropy(fmin(sc * fmax(cc + half, 0.0), 0.36787944117144233));
        }
        acc += contrib;
        wsum += W;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, off);
        wsum += __shfl_xor_sync(0xffffffffu, wsum, off);
        errb += __shfl_xor_sync(0xffffffffu, errb, off);
    }
    if (!(errb <= 1e-10 * fabs(acc))) {
        if (lane == 0) S.fallback = 1;
    } else if (lane == 0) {
        // the weights sum to one; dividing by the computed sum removes their
        // common rounding
        psi[c] = norm2[c] * (acc / wsum);
    }
    __syncwarp();
    if (S.fallback) quad_by_qr<MAXM>(sa, sb, n, sc, norm2[c], lane, psi + c);
}

// f(T) e1 by the sequential implicit QR with the full eigenvector matrix Z
// (n x n, row-major, in shared memory): every lane runs the scalar
// recurrence on its own copies (uniform control flow) and rotates the rows of
// Z it owns (rows lane, lane + 32, ...).  Fallback of k_tridiag_fvec.
template <int MAXM>
__device__ void fvec_by_qr(const double* sa, const double* sb, int n, int m, double sc, int lane, double* Z,
                           double* __restrict__ zvec, int ld, int c) {
    constexpr int R = MAXM / 32;
    for (int idx = lane; idx < n * n; idx += 32) Z[idx] = ((idx / n) == (idx % n)) ? 1.0 : 0.0;
    double dl[MAXM], el[MAXM];
    for (int j = 0; j < n; j++) {
        dl[j] = sa[j];
        el[j] = sb[j];
    }
    double* rows[R];
    int nr = 0;
    for (int q = 0; q < R; q++) {
        const int row = lane + 32 * q;
        rows[q] = Z + (size_t)(row < n ? row : 0) * n;
        if (row < n) nr = q + 1;
    }
    __syncwarp();
    const bool ok = symtri_qr_rows<R>(dl, el, n, rows, nr);
    __syncwarp();
    for (int row = lane; row < m; row += 32) {
        double acc = 0.0;
        if (row < n)
            for (int k = 0; k < n; k++) acc += Z[row * n + k] * f_entropy(sc * dl[k]) * Z[k];
        zvec[(size_t)row * ld + c] = ok ? acc : nan("");
    }
}

// f(T) e1 = sum_j u_j u_{1j} f(sigma theta_j) for the matrix-function
// recovery of the Hutch++ sketch (eq. rational-krylov-approximation-matvec),
// with the spectrum of k_tridiag_quad: an isolated eigenvalue adds its
// twisted-factorisation eigenvector z scaled by z_1 f / ||z||^2; a cluster
// adds (1/2 pi i) \oint (f(c) + f'(c)(z - c) + f''(c)(z - c)^2 / 2)
// (z I - T)^{-1} e1 dz by the 32-point trapezoid rule (one point per lane;
// the resolvent vector from the bottom-up continued fraction, then the
// forward ratios x_k = x_{k-1} beta_{k-1} / g_k).  Each lane accumulates its
// own column of a [n][32] buffer, summed in lane order at the end.
template <int MAXM>
__global__ void __launch_bounds__(32) k_tridiag_fvec(const double* __restrict__ alpha,
                                                     const double* __restrict__ beta,
                                                     const double* __restrict__ scale, int count, int m, int ld,
                                                     double* __restrict__ zvec) {
    __shared__ TqShared<MAXM> S;
    extern __shared__ double piv[];  // [2][MAXM][32] pivots / resolvent, [MAXM][32] partial sums
    const int c = blockIdx.x, lane = threadIdx.x;
    if (c >= count) return;
    if (!tq_spectrum<MAXM>(alpha, beta, c, m, ld, lane, S)) {
        for (int row = lane; row < m; row += 32) zvec[(size_t)row * ld + c] = nan("");
        return;
    }
    const int n = S.n;
    const double span = S.span, pivmin = S.pivmin;
    const double* sa = S.a;
    const double* sb = S.b;
    const double* sth = S.th;
    const double sc = scale[c] / S.s2;  // f is applied to the unscaled eigenvalues
    if (S.fallback) {
        fvec_by_qr<MAXM>(sa, sb, n, m, sc, lane, piv, zvec, ld, c);
        return;
    }
    double* Dp = piv + lane;                // this lane's pivots / real parts
    double* Rp = piv + MAXM * 32 + lane;    // this lane's pivots / imaginary parts
    double* ys = piv + 2 * MAXM * 32 + lane;  // this lane's partial sum of y
    for (int k = 0; k < n; k++) ys[k * 32] = 0.0;
    // isolated eigenvalues
    for (int g = lane; g < S.ngroups; g += 32) {
        if (S.cl_of_group[g] >= 0) continue;
        const double th = sth[S.gfirst[g]];
        double d = 0.0;
        for (int k = 0; k < n; k++) {
            d = guard_pivot((sa[k] - th) - (k > 0 ? sb[k - 1] * sb[k - 1] / d : 0.0), pivmin);
            Dp[k * 32] = d;
        }
        double r = 0.0, best = INFINITY;
        int tw = n - 1;
        for (int k = n - 1; k >= 0; k--) {
            r = guard_pivot((sa[k] - th) - (k + 1 < n ? sb[k] * sb[k] / r : 0.0), pivmin);
            Rp[k * 32] = r;
            const double gam = fabs(Dp[k * 32] + r - (sa[k] - th));
            if (gam < best) {
                best = gam;
                tw = k;
            }
        }
        // eigenvector components overwrite the pivots they were made from
        double nrm = 1.0, z = 1.0;
        for (int k = tw - 1; k >= 0; k--) {
            z = -sb[k] * z / Dp[k * 32];
            Dp[k * 32] = z;
            nrm = fma(z, z, nrm);
        }
        const double z1 = tw > 0 ? z : 1.0;
        z = 1.0;
        for (int k = tw + 1; k < n; k++) {
            z = -sb[k - 1] * z / Rp[k * 32];
            Rp[k * 32] = z;
            nrm = fma(z, z, nrm);
        }
        const double coef = z1 * f_entropy(sc * th) / nrm;
        for (int k = 0; k < n; k++) {
            const double zk = k < tw ? Dp[k * 32] : (k == tw ? 1.0 : Rp[k * 32]);
            ys[k * 32] += coef * zk;
        }
    }
    // clusters: one round per cluster, contour point q on lane q
    double errb = 0.0;
    for (int cl = 0; cl < S.ncl; cl++) {
        const double cc = S.cc[cl], rho = S.rho[cl], half = S.half[cl];
        double sph, cph;
        sincospi((2.0 * lane + 1.0) / kContourPoints, &sph, &cph);
        const double dzr = rho * cph, dzi = rho * sph;
        const double zr = cc + dzr, zi = dzi;
        // bottom-up continued fraction g_k, stored
        double gr = zr - sa[n - 1], gi = zi;
        Dp[(n - 1) * 32] = gr;
        Rp[(n - 1) * 32] = gi;
        for (int k = n - 2; k >= 0; k--) {
            const double t = sb[k] * sb[k] / (gr * gr + gi * gi);
            gr = (zr - sa[k]) - t * gr;
            gi = zi + t * gi;
            Dp[k * 32] = gr;
            Rp[k * 32] = gi;
        }
        // Taylor weight h = dz (f0 + f1 dz + f2 dz^2 / 2) of the cluster centre
        const double x0 = sc * cc;
        const double f0 = f_entropy(x0);
        const double f1 = x0 > 0.0 ? sc * (-log(x0) - 1.0) : 0.0;
        const double f2 = cc > 0.0 ? -sc / cc : 0.0;
        const double d2r = dzr * dzr - dzi * dzi, d2i = 2.0 * dzr * dzi;
        const double pr = f0 + f1 * dzr + 0.5 * f2 * d2r, pi = f1 * dzi + 0.5 * f2 * d2i;
        const double hr = (dzr * pr - dzi * pi) / kContourPoints, hi = (dzr * pi + dzi * pr) / kContourPoints;
        // forward ratios: x_0 = 1 / g_0, x_k = x_{k-1} beta_{k-1} / g_k
        double xr, xi;
        {
            const double den = gr * gr + gi * gi;
            xr = gr / den;
            xi = -gi / den;
        }
        double wq = (xr * dzr - xi * dzi) / kContourPoints;  // Re x_0 dz / K
        ys[0] += xr * hr - xi * hi;
        for (int k = 1; k < n; k++) {
            const double g_r = Dp[k * 32], g_i = Rp[k * 32];
            const double den = g_r * g_r + g_i * g_i;
            const double ur = sb[k - 1] * g_r / den, ui = -sb[k - 1] * g_i / den;  // beta / g
            const double nxr = xr * ur - xi * ui, nxi = xr * ui + xi * ur;
            xr = nxr;
            xi = nxi;
            ys[k * 32] += xr * hr - xi * hi;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) wq += __shfl_xor_sync(0xffffffffu, wq, off);
        if (half > 1e-3 * fabs(cc))  // cluster at the origin: error below W f(c + half)
            errb += fmax(wq, 0.0) * f_entropy(fmin(sc * fmax(cc + half, 0.0), 0.36787944117144233));
    }
    __syncwarp();
    // y_k = sum over lanes of the partial sums, in lane order
    double y0 = 0.0;
    for (int k = lane; k < m; k += 32) {
        double y = 0.0;
        if (k < n)
            for (int l = 0; l < 32; l++) y += piv[2 * MAXM * 32 + k * 32 + l];
        if (k == 0) y0 = y;
        zvec[(size_t)k * ld + c] = y;
    }
    y0 = __shfl_sync(0xffffffffu, y0, 0);
    if (!(errb <= 1e-10 * fabs(y0))) {
        __syncwarp();
        fvec_by_qr<MAXM>(sa, sb, n, m, sc, lane, piv, zvec, ld, c);
    }
}

// A-posteriori bounds of Theorem 4.4 for the polynomial Lanczos quadrature
// after m steps (A V_m = V_m T_m + beta_m v_{m+1} e_m^T): with Ritz values
// theta_j, a_j = beta_m U_{mj}, b_j = U_{1j} and
// gamma_j = sum_{l != j} a_l b_l / (theta_j - theta_l),
//   g_m(z) = sum_j a_j^2 b_j^2 f[theta_j, theta_j, z] + 2 a_j b_j gamma_j f[theta_j, z]
// (divided differences of f, the limits at z = theta_j included; evaluated
// stably, see dd_entropy), and ||c||^2 min / max of |g_m| over the
// spectral interval bound the quadrature error from below / above; their
// geometric mean is the paper's error estimate.  The minimum and maximum are
// taken over `grid` geometrically and `grid` linearly spaced points of
// [lam_min, lam_max] plus the Ritz values inside it, spread over the lanes.
// U_{1j}, U_{mj} come from the twisted-factorisation eigenvectors of the
// shared spectrum (for a tight cluster the individual products are as
// ill-conditioned as the formula itself).  f(x) = -x log x; the interval must
// be positive.
// Divided differences of f(x) = -x log x at (t, z), z = t (1 + u), given
// log z and log t: f[t, z] = -log t - h(u) and f[t, t, z] = (1 - h(u)) / (t u)
// with h(u) = (1 + u) log(1 + u) / u = z (log z - log t) / (t u).  For
// |u| < 0.1 the power series 1 - h(u) = sum_{k>=1} (-1)^k u^k / (k (k + 1))
// avoids the cancellation of the plain quotients.
__device__ __forceinline__ void dd_entropy(double z, double lz, double t, double lt, double& dd1, double& dd2) {
    const double u = (z - t) / t;
    if (fabs(u) < 0.1) {
        // (1 - h(u)) / u by Horner, 18 terms (|u|^18 / 342 < 1e-20)
        double ser = 0.0;
        for (int k = 18; k >= 1; k--) ser = fma(ser, u, ((k & 1) ? -1.0 : 1.0) / (double)(k * (k + 1)));
        dd1 = -lt - (1.0 - ser * u);
        dd2 = ser / t;
    } else {
        const double h = (z / t) * (lz - lt) / u;
        dd1 = -lt - h;
        dd2 = (1.0 - h) / (t * u);
    }
}

template <int MAXM>
__global__ void __launch_bounds__(32) k_tridiag_bounds(const double* __restrict__ alpha,
                                                       const double* __restrict__ beta,
                                                       const double* __restrict__ norm2,
                                                       const double* __restrict__ scale, int count, int m_all, int ld,
                                                       double lam_min, double lam_max, int grid,
                                                       double* __restrict__ lower, double* __restrict__ upper,
                                                       double* __restrict__ estimate,
                                                       const int32_t* __restrict__ cols,
                                                       const int32_t* __restrict__ mcol,
                                                       const double* __restrict__ lam_max_col) {
    __shared__ TqShared<MAXM> S;
    __shared__ double s_th[MAXM], s_ab[MAXM], s_gam[MAXM], s_lt[MAXM];
    extern __shared__ double piv[];  // [2][MAXM][32] twisted pivots
    const int lane = threadIdx.x;
    if ((int)blockIdx.x >= count) return;
    // entry blockIdx.x: column c (of the ld-strided arrays) after m steps,
    // with its own upper end of the spectral interval if given
    const int c = cols ? cols[blockIdx.x] : (int)blockIdx.x;
    const int m = mcol ? mcol[blockIdx.x] : m_all;
    if (lam_max_col) lam_max = lam_max_col[blockIdx.x];
    if (!tq_spectrum<MAXM>(alpha, beta, c, m, ld, lane, S)) {
        if (lane == 0) lower[c] = upper[c] = estimate[c] = nan("");
        return;
    }
    const int n = S.n;
    const double bm = beta[(size_t)(m - 1) * ld + c] * scale[c];  // beta_m of A
    if (n < m || bm == 0.0) {
        // the Krylov space is invariant: the quadrature is exact
        if (lane == 0) lower[c] = upper[c] = estimate[c] = 0.0;
        return;
    }
    const double sc = scale[c] / S.s2;
    double* Dp = piv + lane;
    double* Rp = piv + MAXM * 32 + lane;
    // first and last eigenvector components
    for (int j = lane; j < n; j += 32) {
        const double th = S.th[j];
        double d = 0.0;
        for (int k = 0; k < n; k++) {
            d = guard_pivot((S.a[k] - th) - (k > 0 ? S.b[k - 1] * S.b[k - 1] / d : 0.0), S.pivmin);
            Dp[k * 32] = d;
        }
        double r = 0.0, best = INFINITY;
        int tw = n - 1;
        for (int k = n - 1; k >= 0; k--) {
            r = guard_pivot((S.a[k] - th) - (k + 1 < n ? S.b[k] * S.b[k] / r : 0.0), S.pivmin);
            Rp[k * 32] = r;
            const double gam = fabs(Dp[k * 32] + r - (S.a[k] - th));
            if (gam < best) {
                best = gam;
                tw = k;
            }
        }
        double nrm = 1.0, z = 1.0;
        for (int k = tw - 1; k >= 0; k--) {
            z = -S.b[k] * z / Dp[k * 32];
            nrm = fma(z, z, nrm);
        }
        const double z1 = tw > 0 ? z : 1.0;
        z = 1.0;
        for (int k = tw + 1; k < n; k++) {
            z = -S.b[k - 1] * z / Rp[k * 32];
            nrm = fma(z, z, nrm);
        }
        const double zn = tw < n - 1 ? z : 1.0;
        s_th[j] = sc * th;
        s_ab[j] = bm * (zn * z1) / nrm;
    }
    __syncwarp();
    for (int j = lane; j < n; j += 32) {
        const double t = s_th[j];
        double gsum = 0.0;
        for (int l = 0; l < n; l++)
            if (l != j) gsum += s_ab[l] / (t - s_th[l]);
        s_gam[j] = gsum;
        s_lt[j] = log(t);
    }
    __syncwarp();
    if (!(lam_min > 0.0)) {
        // half the smallest positive Ritz value of this column
        double tmin = INFINITY;
        for (int j = lane; j < n; j += 32)
            if (s_th[j] > 0.0) tmin = fmin(tmin, s_th[j]);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) tmin = fmin(tmin, __shfl_xor_sync(0xffffffffu, tmin, off));
        lam_min = 0.5 * tmin;
    }
    if (!(lam_min > 0.0 && lam_max > lam_min)) {
        if (lane == 0) lower[c] = upper[c] = estimate[c] = INFINITY;  // no usable interval: not converged
        return;
    }
    const int npts = 2 * grid + n;
    const double lratio = log(lam_max / lam_min);
    double gmin = INFINITY, gmax = 0.0;
    for (int q = lane; q < npts; q += 32) {
        double z;
        if (q < grid) z = grid > 1 ? lam_min * exp(lratio * q / (grid - 1)) : lam_min;
        else if (q < 2 * grid) z = grid > 1 ? lam_min + (lam_max - lam_min) * (q - grid) / (grid - 1) : lam_min;
        else {
            z = s_th[q - 2 * grid];
            if (!(z >= lam_min && z <= lam_max)) continue;
        }
        const double lz = log(z);
        double g = 0.0;
        for (int j = 0; j < n; j++) {
            const double ab = s_ab[j];
            double dd1, dd2;
            dd_entropy(z, lz, s_th[j], s_lt[j], dd1, dd2);
            g += ab * ab * dd2 + 2.0 * ab * s_gam[j] * dd1;
        }
        gmin = fmin(gmin, fabs(g));
        gmax = fmax(gmax, fabs(g));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        gmin = fmin(gmin, __shfl_xor_sync(0xffffffffu, gmin, off));
        gmax = fmax(gmax, __shfl_xor_sync(0xffffffffu, gmax, off));
    }
    if (lane == 0) {
        const double nb = norm2[c];
        lower[c] = nb * gmin;
        upper[c] = nb * gmax;
        estimate[c] = nb * sqrt(gmin * gmax);
    }
}

cudaError_t launch_tridiag_bounds(const double* alpha, const double* beta, const double* norm2, const double* scale,
                                  int count, int m, int ld, double lam_min, double lam_max, int grid, double* lower,
                                  double* upper, double* estimate, cudaStream_t st) {
    return launch_tridiag_bounds_list(alpha, beta, norm2, scale, count, nullptr, nullptr, nullptr, m, ld, lam_min,
                                      lam_max, grid, lower, upper, estimate, st);
}

cudaError_t launch_tridiag_bounds_list(const double* alpha, const double* beta, const double* norm2,
                                       const double* scale, int count, const int32_t* cols, const int32_t* mcol,
                                       const double* lam_max_col, int m, int ld, double lam_min, double lam_max,
                                       int grid, double* lower, double* upper, double* estimate, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    // lam_min <= 0: half the smallest positive Ritz value of each column
    if ((!lam_max_col && !(lam_max > 0.0 && lam_max > lam_min)) || grid < 1) return cudaErrorInvalidValue;
#define VNE_BOUND_CASE(MM)                                                                                   \
    if (m <= MM) {                                                                                          \
        const int smem = 2 * MM * 32 * (int)sizeof(double);                                                 \
        cudaError_t e = cudaFuncSetAttribute(k_tridiag_bounds<MM>,                                          \
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);            \
        if (e != cudaSuccess) return e;                                                                     \
        k_tridiag_bounds<MM><<<count, 32, smem, st>>>(alpha, beta, norm2, scale, count, m, ld, lam_min, lam_max, \
                                                       grid, lower, upper, estimate, cols, mcol, lam_max_col); \
        return cudaGetLastError();                                                                          \
    }
    VNE_BOUND_CASE(32)
    VNE_BOUND_CASE(64)
    VNE_BOUND_CASE(128)
#undef VNE_BOUND_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_tridiag_quad(const double* alpha, const double* beta, const double* norm2,
                                const double* scale_per_col, int count, int m, int ld, double* psi,
                                cudaStream_t st) {
    return launch_tridiag_quad_list(alpha, beta, norm2, scale_per_col, count, nullptr, nullptr, m, ld, psi, st);
}

cudaError_t launch_tridiag_quad_list(const double* alpha, const double* beta, const double* norm2,
                                     const double* scale_per_col, int count, const int32_t* cols,
                                     const int32_t* mcol, int m, int ld, double* psi, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    // one warp (CTA) per tridiagonal; dynamic shared memory holds the
    // twisted-factorisation pivots of the 32 lanes
#define VNE_QUAD_CASE(MM)                                                                                    \
    if (m <= MM) {                                                                                          \
        const int smem = 2 * MM * 32 * (int)sizeof(double);                                                 \
        cudaError_t e = cudaFuncSetAttribute(k_tridiag_quad<MM>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                             smem);                                                         \
        if (e != cudaSuccess) return e;                                                                     \
        k_tridiag_quad<MM><<<count, 32, smem, st>>>(alpha, beta, norm2, scale_per_col, count, m, ld, psi,    \
                                                     cols, mcol);                                           \
        return cudaGetLastError();                                                                          \
    }
    VNE_QUAD_CASE(32)
    VNE_QUAD_CASE(64)
    VNE_QUAD_CASE(128)
#undef VNE_QUAD_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_tridiag_fvec(const double* alpha, const double* beta, const double* scale_per_col, int count,
                                int m, int ld, double* zvec, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    // one warp (CTA) per tridiagonal; dynamic shared memory: pivots /
    // resolvent and the lanes' partial sums (3 x MM x 32 doubles), or Z for
    // the QR fallback (MM x MM)
#define VNE_FVEC_CASE(MM)                                                                                    \
    if (m <= MM) {                                                                                          \
        const int words = 3 * MM * 32 > MM * MM ? 3 * MM * 32 : MM * MM;                                    \
        const int smem = words * (int)sizeof(double);                                                       \
        cudaError_t e = cudaFuncSetAttribute(k_tridiag_fvec<MM>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                             smem);                                                         \
        if (e != cudaSuccess) return e;                                                                     \
        k_tridiag_fvec<MM><<<count, 32, smem, st>>>(alpha, beta, scale_per_col, count, m, ld, zvec);         \
        return cudaGetLastError();                                                                          \
    }
    VNE_FVEC_CASE(32)
    VNE_FVEC_CASE(64)
    VNE_FVEC_CASE(128)
#undef VNE_FVEC_CASE
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Gram C = X^T Y, 64 x 64 output tile per CTA, rows split into chunks.
// Each thread owns a 4 x 4 block of the tile; the 64-row slabs of X and Y are
// staged transposed-free in shared memory ([row][col], float4-aligned).
// Products accumulate in the data precision over one 64-row slab, then in
// FP64 across slabs.
template <typename T, int KS>
__global__ void __launch_bounds__(256) k_gram(const T* __restrict__ X, int kx, const T* __restrict__ Y, int ky,
                                              int n, int rows_per_chunk, int tiles_y, double* __restrict__ part) {
    __shared__ __align__(16) T Xs[64][64];
    __shared__ __align__(16) T Ys[64][64];
    const int chunk = blockIdx.x;
    const int tx0 = (blockIdx.y / tiles_y) * 64, ty0 = (blockIdx.y % tiles_y) * 64;
    const int r_begin = chunk * rows_per_chunk;
    const int r_end = min(n, r_begin + rows_per_chunk);
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double dacc[4][4];
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) dacc[a][b] = 0.0;
    for (int rt = r_begin; rt < r_end; rt += 64) {
        // each panel row holds KS consecutive columns: copy whole KS-runs
        for (int idx = threadIdx.x; idx < 64 * 64; idx += 256) {
            int rl = idx / 64, cl = idx % 64;
            int r = rt + rl;
            int cxg = tx0 + cl, cyg = ty0 + cl;
            T xv = (T)0, yv = (T)0;
            if (r < r_end) {
                if (cxg < kx) xv = X[(size_t)(cxg / KS) * n * KS + (size_t)r * KS + (cxg % KS)];
                if (cyg < ky) yv = Y[(size_t)(cyg / KS) * n * KS + (size_t)r * KS + (cyg % KS)];
            }
            Xs[rl][cl] = xv;
            Ys[rl][cl] = yv;
        }
        __syncthreads();
        T acc[4][4];
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int b = 0; b < 4; b++) acc[a][b] = (T)0;
#pragma unroll 4
        for (int rl = 0; rl < 64; rl++) {
            T xa[4], yb[4];
#pragma unroll
            for (int a = 0; a < 4; a++) xa[a] = Xs[rl][tx * 4 + a];
#pragma unroll
            for (int b = 0; b < 4; b++) yb[b] = Ys[rl][ty * 4 + b];
#pragma unroll
            for (int a = 0; a < 4; a++)
#pragma unroll
                for (int b = 0; b < 4; b++) acc[a][b] += xa[a] * yb[b];
        }
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int b = 0; b < 4; b++) dacc[a][b] += (double)acc[a][b];
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) {
            int i = tx0 + tx * 4 + a, j = ty0 + ty * 4 + b;
            if (i < kx && j < ky) part[(size_t)chunk * kx * ky + (size_t)i * ky + j] = dacc[a][b];
        }
}

__global__ void k_gram_reduce(const double* __restrict__ part, int nchunks, int total, double* __restrict__ C) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    double s = 0.0;
    for (int c = 0; c < nchunks; c++) s += part[(size_t)c * total + idx];
    C[idx] = s;
}

// C <- C + C^T in place (C = the summed partials E of a symmetric Gram): one
// thread per pair a <= b.
__global__ void k_gram_symmetrize(double* __restrict__ C, int k) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= k * k) return;
    const int a = idx / k, b = idx % k;
    if (a > b) return;
    const double s = C[a * k + b] + C[b * k + a];
    C[a * k + b] = s;
    C[b * k + a] = s;
}

template <typename T>
cudaError_t launch_gram(const T* X, int kx, const T* Y, int ky, int ks, int n, double* part, int nchunks, double* C,
                        int* err, cudaStream_t st) {
    if (kx <= 0 || ky <= 0) return cudaSuccess;
    if (sizeof(T) == 4 && err && kx <= 128 && ky <= 128 && (ks == 8 || ks == 16 || ks == 32)) {
        int chunks = 0, sym = 0;
        cudaError_t e = launch_gram_tc5(reinterpret_cast<const float*>(X), kx, reinterpret_cast<const float*>(Y), ky,
                                        ks, n, part, nchunks, err, &chunks, &sym, st);
        if (e != cudaSuccess) return e;
        const int total = kx * ky;
        k_gram_reduce<<<(total + 255) / 256, 256, 0, st>>>(part, chunks, total, C);
        if (sym) k_gram_symmetrize<<<(total + 255) / 256, 256, 0, st>>>(C, kx);
        return cudaGetLastError();
    }
    int tiles_x = (kx + 63) / 64, tiles_y = (ky + 63) / 64;
    int rpc = (n + nchunks - 1) / nchunks;
    rpc = ((rpc + 63) / 64) * 64;
    int chunks = rpc > 0 ? (n + rpc - 1) / rpc : 1;
    if (chunks < 1) chunks = 1;
    dim3 grid(chunks, tiles_x * tiles_y);
    if (ks == 4) k_gram<T, 4><<<grid, 256, 0, st>>>(X, kx, Y, ky, n, rpc, tiles_y, part);
    else if (ks == 8) k_gram<T, 8><<<grid, 256, 0, st>>>(X, kx, Y, ky, n, rpc, tiles_y, part);
    else if (ks == 16) k_gram<T, 16><<<grid, 256, 0, st>>>(X, kx, Y, ky, n, rpc, tiles_y, part);
    else if (ks == 32) k_gram<T, 32><<<grid, 256, 0, st>>>(X, kx, Y, ky, n, rpc, tiles_y, part);
    else return cudaErrorInvalidValue;
    int total = kx * ky;
    k_gram_reduce<<<(total + 255) / 256, 256, 0, st>>>(part, chunks, total, C);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Out = In2 + coef * In * M.  Persistent CTAs: M (FP64 [kin][kout]) is staged
// once per CTA in shared memory in the data precision, then 64-row tiles of
// In are streamed through shared memory (stored transposed, [k][row]); each
// thread owns 4 rows x 8 output columns.
template <typename T, int KS>
__global__ void __launch_bounds__(256) k_apply(const T* __restrict__ In, int kin, const double* __restrict__ M,
                                               int kout, const T* __restrict__ In2, T* __restrict__ Out, int n,
                                               double coef) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T* Ms = reinterpret_cast<T*>(smraw);          // [kin][128]
    T* Ist = Ms + (size_t)kin * 128;              // [kin][64]  (transposed tile)
    for (int idx = threadIdx.x; idx < kin * 128; idx += 256) {
        int a = idx / 128, b = idx % 128;
        Ms[idx] = (b < kout) ? (T)(coef * M[(size_t)a * kout + b]) : (T)0;
    }
    const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;  // rows ty*4.., cols tx*8..
    const int ntiles = (n + 63) / 64;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int r0 = tile * 64;
        __syncthreads();
        for (int idx = threadIdx.x; idx < 64 * kin; idx += 256) {
            int c = idx / 64, rl = idx % 64;
            int r = r0 + rl;
            Ist[idx] = (r < n) ? In[(size_t)(c / KS) * n * KS + (size_t)r * KS + (c % KS)] : (T)0;
        }
        __syncthreads();
        if (tx * 8 >= kout) continue;
        T acc[4][8];
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int b = 0; b < 8; b++) acc[a][b] = (T)0;
        for (int k = 0; k < kin; k++) {
            T av[4], bv[8];
#pragma unroll
            for (int a = 0; a < 4; a++) av[a] = Ist[k * 64 + ty * 4 + a];
#pragma unroll
            for (int b = 0; b < 8; b++) bv[b] = Ms[k * 128 + tx * 8 + b];
#pragma unroll
            for (int a = 0; a < 4; a++)
#pragma unroll
                for (int b = 0; b < 8; b++) acc[a][b] += av[a] * bv[b];
        }
#pragma unroll
        for (int a = 0; a < 4; a++) {
            const int r = r0 + ty * 4 + a;
            if (r >= n) continue;
#pragma unroll
            for (int b = 0; b < 8; b++) {
                const int c = tx * 8 + b;
                if (c < kout) {
                    size_t o = (size_t)(c / KS) * n * KS + (size_t)r * KS + (c % KS);
                    T v = acc[a][b];
                    if (In2) v += In2[o];
                    Out[o] = v;
                }
            }
        }
    }
}

template <typename T>
cudaError_t launch_apply(const T* In, int kin, const double* M, int kout, const T* In2, T* Out, int ks, int n,
                         double coef, int* err, cudaStream_t st) {
    if (kout > 128 || kin > 128) return cudaErrorInvalidValue;
    if (sizeof(T) == 4 && err && kin > 0 && kout > 0 && (ks == 8 || ks == 16 || ks == 32))
        return launch_apply_tc5(reinterpret_cast<const float*>(In), kin, M, kout, reinterpret_cast<const float*>(In2),
                                reinterpret_cast<float*>(Out), ks, n, coef, err, st);
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int ntiles = (n + 63) / 64;
    size_t smem = ((size_t)kin * 128 + 64 * (size_t)kin) * sizeof(T);
    int per_sm = sizeof(T) == 4 ? 2 : 1;
    dim3 grid(ntiles < sms * per_sm ? ntiles : sms * per_sm);
#define VNE_APPLY_CASE(KSV)                                                                                  \
    if (ks == KSV) {                                                                                        \
        cudaError_t e = cudaFuncSetAttribute(k_apply<T, KSV>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                             (int)smem);                                                    \
        if (e != cudaSuccess) return e;                                                                     \
        k_apply<T, KSV><<<grid, 256, smem, st>>>(In, kin, M, kout, In2, Out, n, coef);                      \
        return cudaGetLastError();                                                                          \
    }
    VNE_APPLY_CASE(4)
    VNE_APPLY_CASE(8)
    VNE_APPLY_CASE(16)
    VNE_APPLY_CASE(32)
#undef VNE_APPLY_CASE
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Pivoted Cholesky G = P R^T R P^T (FP64), in two kernels: the factor (one
// CTA) and the triangular inverse (a warp per column).  Stops when the
// largest remaining pivot is <= tol * max diag(G); rank r = pivots taken.
// Writes Minv with Minv[piv[i]][c] = (R^{-1})[i][c] for i, c < r, zero
// elsewhere, so that Y Minv has orthonormal columns in exact arithmetic.
// Pivoted Cholesky factor of the FP64 Gram (one CTA): R upper triangular
// with P^T G P = R^T R, the pivots, 1 / R_jj and the numerical rank (the
// first pivot below tol * max diag stops the factorisation).  FP64 runs at a
// small fraction of the FP32 rate on this part, so a step costs one square
// root and one reciprocal (thread 0) and the row is scaled by multiplication.
// Output R: work[0 .. k*k) row-major (upper triangle), 1 / R_jj:
// work[k*k .. k*k + k), pivots: piv[0 .. k).  With pivot = 0 the columns are
// taken in their order (plain Cholesky; the first pivot below the cut-off
// stops it).
__global__ void k_chol_factor(const double* __restrict__ G, int k, double tol, double* __restrict__ work,
                              int* __restrict__ piv_out, int* __restrict__ rank_out, int pivot) {
    extern __shared__ double A[];  // k x (k + 1): odd row stride against bank conflicts
    const int ld = k + 1;
    __shared__ int piv[128];
    __shared__ int s_p, s_rank;
    __shared__ double s_max0, s_rinv;
    // symmetric part of G (the Gram partial sums of (a, b) and (b, a) may
    // round differently)
    for (int idx = threadIdx.x; idx < k * k; idx += blockDim.x) {
        const int a = idx / k, b = idx % k;
        A[a * ld + b] = 0.5 * (G[idx] + G[b * k + a]);
    }
    for (int i = threadIdx.x; i < k; i += blockDim.x) piv[i] = i;
    __syncthreads();
    if (threadIdx.x == 0) {
        double mx = 0.0;
        for (int i = 0; i < k; i++) mx = fmax(mx, A[i * ld + i]);
        s_max0 = mx;
        s_rank = k;
    }
    __syncthreads();
    for (int j = 0; j < k; j++) {
        if (threadIdx.x < 32) {
            // largest remaining diagonal entry (warp argmax, ties to the lower index)
            double best = -INFINITY;
            int p = j;
            if (pivot) {
                for (int i = j + (int)threadIdx.x; i < k; i += 32)
                    if (A[i * ld + i] > best) {
                        best = A[i * ld + i];
                        p = i;
                    }
            } else if (threadIdx.x == 0) {
                best = A[j * ld + j];
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, off);
                const int op = __shfl_xor_sync(0xffffffffu, p, off);
                if (ob > best || (ob == best && op < p)) {
                    best = ob;
                    p = op;
                }
            }
            if (threadIdx.x == 0) {
                s_p = (best > tol * s_max0 && best > 0.0) ? p : -1;
                if (s_p < 0) s_rank = j;
            }
        }
        __syncthreads();
        const int p = s_p;
        if (p < 0) break;
        if (p != j) {
            for (int i = threadIdx.x; i < k; i += blockDim.x) {  // swap rows
                double t = A[j * ld + i];
                A[j * ld + i] = A[p * ld + i];
                A[p * ld + i] = t;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < k; i += blockDim.x) {  // swap columns
                double t = A[i * ld + j];
                A[i * ld + j] = A[i * ld + p];
                A[i * ld + p] = t;
            }
            if (threadIdx.x == 0) {
                int t = piv[j];
                piv[j] = piv[p];
                piv[p] = t;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const double rjj = sqrt(A[j * ld + j]);
            A[j * ld + j] = rjj;
            s_rinv = 1.0 / rjj;
        }
        __syncthreads();
        const double rinv = s_rinv;
        for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x) A[j * ld + i] *= rinv;
        if (threadIdx.x == 0) work[(size_t)k * k + j] = rinv;
        __syncthreads();
        // rank-1 update of the trailing block: the upper triangle (a warp per
        // row), mirrored into the lower one for later pivot swaps
        const int rem = k - j - 1;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
        for (int a = warp; a < rem; a += nwarp) {
            const int ga = j + 1 + a;
            const double la = A[j * ld + ga];
            for (int gb = ga + lane; gb < k; gb += 32) {
                const double v = fma(-la, A[j * ld + gb], A[ga * ld + gb]);
                A[ga * ld + gb] = v;
                A[gb * ld + ga] = v;
            }
        }
        __syncthreads();
    }
    __syncthreads();
    const int r = s_rank;
    for (int idx = threadIdx.x; idx < k * k; idx += blockDim.x) {
        const int a = idx / k, b = idx % k;
        work[idx] = (a < r && b >= a) ? A[a * ld + b] : 0.0;
    }
    for (int i = threadIdx.x; i < k; i += blockDim.x) piv_out[i] = piv[i];
    if (threadIdx.x == 0) *rank_out = r;
}

// Minv = P R^{-1} (rows permuted back), zero beyond the rank: column c of
// R^{-1} by back substitution, x_c = 1 / R_cc and, for i = c - 1 .. 0,
// x_i = -(sum_{l = i+1..c} R_il x_l) / R_ii.  One warp per column, R staged
// in shared memory, the inner products lane-parallel with a butterfly sum;
// the columns are spread over the SMs (a column's chain is serial).
__global__ void __launch_bounds__(256) k_tri_inv(const double* __restrict__ work, int k, const int* __restrict__ piv,
                                                 const int* __restrict__ rank, double* __restrict__ Minv) {
    extern __shared__ double R[];  // rows 0 .. c_hi of R, row stride k + 1
    __shared__ double xs[8][128];
    const int ld = k + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = *rank;
    const int c_hi = min(k - 1, (int)blockIdx.x * 8 + 7);  // last column of this CTA
    for (int idx = threadIdx.x; idx < (c_hi + 1) * k; idx += blockDim.x) {
        const int a = idx / k, b = idx % k;
        R[a * ld + b] = work[idx];
    }
    __syncthreads();
    const int c = blockIdx.x * 8 + warp;
    if (c >= k) return;
    const double* rinv = work + (size_t)k * k;
    double* x = xs[warp];
    if (c < r) {
        if (lane == 0) x[c] = rinv[c];
        __syncwarp();
        for (int i = c - 1; i >= 0; i--) {
            double s = 0.0;
            for (int l = i + 1 + lane; l <= c; l += 32) s = fma(R[i * ld + l], x[l], s);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            if (lane == 0) x[i] = -s * rinv[i];
            __syncwarp();
        }
    }
    for (int i = lane; i < k; i += 32) Minv[(size_t)piv[i] * k + c] = (c < r && i <= c) ? x[i] : 0.0;
}

cudaError_t launch_chol_qr_factor(const double* G, int k, double tol, double* Minv, int* rank, double* work,
                                  int* piv, cudaStream_t st, bool pivot) {
    if (k > 128 || k <= 0) return cudaErrorInvalidValue;
    const size_t smem = (size_t)k * (k + 1) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_chol_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_tri_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_chol_factor<<<1, 256, smem, st>>>(G, k, tol, work, piv, rank, pivot ? 1 : 0);
    k_tri_inv<<<(k + 7) / 8, 256, smem, st>>>(work, k, piv, rank, Minv);
    return cudaGetLastError();
}

template cudaError_t launch_gram<float>(const float*, int, const float*, int, int, int, double*, int, double*, int*,
                                       cudaStream_t);
template cudaError_t launch_gram<double>(const double*, int, const double*, int, int, int, double*, int, double*, int*,
                                        cudaStream_t);
template cudaError_t launch_apply<float>(const float*, int, const double*, int, const float*, float*, int, int, double, int*, cudaStream_t);
template cudaError_t launch_apply<double>(const double*, int, const double*, int, const double*, double*, int, int, double, int*, cudaStream_t);

}  // namespace vne
