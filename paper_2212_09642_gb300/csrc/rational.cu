// Rational Krylov quadrature with negative real poles (Sections 4, 4.2, 5.3)
// via a batched multi-shift conjugate gradient.
//
// For poles xi_s = -s_s (s_s > 0) and ell poles at infinity the rational
// Krylov space of eq. rational-krylov-subspace-definition is, by partial
// fractions, span{c, A c, .., A^ell c, x_1, .., x_S} with
// x_s = (A + s_s I)^{-1} c.  All S shifted systems are solved from one
// Krylov sequence: conjugate gradients run on the seed system (A + s_0 I),
// s_0 the smallest shift, and every shifted residual stays collinear with the
// seed residual, r_s = zeta_s r, which gives each shifted iterate from the
// seed's coefficients (Jegerlehner 1996; Frommer 2003).  A shift is retired
// once |zeta_s| ||r|| <= tol ||c||.
//
// Per CG iteration, for a block of K columns (panel-major, as in the
// Lanczos engine):
//   step kernel (shared with Lanczos)  q = (A + s_0 I) p,  d = p . q
//   k_cg_scalars_a   a = rho / d, zeta_{k+1}, a_s     (per column, FP64)
//   k_cg_update      p_s = zeta_k r + b_s p_s, x_s += a_s p_s, r -= a q,
//                    rho' = ||r||^2
//   k_cg_scalars_b   b = rho'/rho, b_s, convergence, shift history
//   k_cg_direction   p = r + b p
// Afterwards the basis W and A W are formed (A^j c by the step kernel,
// A x_s by the step kernel), their Gram matrices W^T W and W^T A W are
// accumulated per column in one pass over the vectors (k_multi_gram), and a per-column FP64 kernel orthonormalises W in
// pole order (Cholesky of the column-scaled Gram, dropping dependent
// columns; the first basis vector is c / ||c|| as in rational Arnoldi),
// applies that basis change to the vectors W and A W and repeats the
// orthonormalisation from the new Gram matrices (Cholesky-QR2, so the
// rounding error no longer grows with the square of the basis condition
// number), projects A, diagonalises the small matrix by cyclic Jacobi and
// returns psi = ||c||^2 e1^T f(A_m) e1.
#include <float.h>
#include <math.h>

#include "common.cuh"
#include "kernels.h"

namespace vne {

constexpr int kMaxShifts = 8;
constexpr int kMaxBasis = 24;  // 1 + up to 15 polynomial directions + 8 poles

__device__ __forceinline__ double f_ent(double x) { return x > 0.0 ? -x * log(x) : 0.0; }

// x_s = 0, r = p = p_s = c are set by copies; here the scalar state:
// rho = ||c||^2, zeta = zeta_prev = 1, a_prev = 1, b_prev = 0, all shifts
// active for non-zero columns.
__global__ void k_cg_init(CgState st, const double* norm2) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= st.K) return;
    const double n2 = norm2[c];
    st.rho[c] = n2;
    st.cnorm[c] = sqrt(n2);
    st.a_prev[c] = 1.0;
    st.b_prev[c] = 0.0;
    st.a[c] = 0.0;
    st.b[c] = 0.0;
    for (int s = 0; s < st.nshift; s++) {
        const size_t o = (size_t)s * st.K + c;
        st.zeta[o] = 1.0;
        st.zeta_prev[o] = 1.0;
        st.zeta_next[o] = 1.0;
        st.as[o] = 0.0;
        st.bs[o] = 0.0;
        st.active[o] = n2 > 0.0 ? 1 : 0;
        st.iters[o] = 0;
        st.resid[o] = n2 > 0.0 ? 1.0 : 0.0;
    }
}

cudaError_t launch_cg_init(CgState st, const double* norm2, cudaStream_t s) {
    k_cg_init<<<(st.K + 63) / 64, 64, 0, s>>>(st, norm2);
    return cudaGetLastError();
}

// per column: a = rho / d (d from the step kernel as scale * (p . q)), then
// the shifted coefficients
__global__ void k_cg_scalars_a(CgState st) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= st.K) return;
    const double d = st.dq[c] / st.scale;
    const double rho = st.rho[c];
    double a = (d > 0.0 && rho > 0.0) ? rho / d : 0.0;
    st.a[c] = a;
    for (int s = 0; s < st.nshift; s++) {
        const size_t o = (size_t)s * st.K + c;
        if (!st.active[o] || a == 0.0) {
            st.as[o] = 0.0;
            continue;
        }
        const double zk = st.zeta[o], zkm1 = st.zeta_prev[o];
        const double ap = st.a_prev[c], bp = st.b_prev[c];
        const double delta = st.shift[s] - st.shift0;
        const double den = ap * zkm1 * (1.0 + delta * a) + a * bp * (zkm1 - zk);
        const double zn = (den != 0.0) ? zk * zkm1 * ap / den : 0.0;
        st.zeta_next[o] = zn;
        st.as[o] = (zk != 0.0) ? a * zn / zk : 0.0;
    }
}

// per column: b = rho' / rho and the shifted b_s, convergence, history shift
__global__ void k_cg_scalars_b(CgState st) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= st.K) return;
    const double rho = st.rho[c], rhon = st.rho_new[c];
    const double b = (rho > 0.0) ? rhon / rho : 0.0;
    st.b[c] = b;
    const double rnorm = sqrt(rhon);
    int any = 0;
    for (int s = 0; s < st.nshift; s++) {
        const size_t o = (size_t)s * st.K + c;
        if (!st.active[o]) continue;
        const double zk = st.zeta[o], zn = st.zeta_next[o];
        const double ratio = (zk != 0.0) ? zn / zk : 0.0;
        st.bs[o] = b * ratio * ratio;
        st.zeta_prev[o] = zk;
        st.zeta[o] = zn;
        st.iters[o] += 1;
        const double res = fabs(zn) * rnorm;
        st.resid[o] = res / st.cnorm[c];
        if (!(res > st.tol * st.cnorm[c])) st.active[o] = 0;  // converged (or breakdown)
        else any = 1;
    }
    st.a_prev[c] = st.a[c];
    st.b_prev[c] = b;
    st.rho[c] = rhon;
    if (any) atomicOr(st.any_active, 1);
}

// r -= a q;  rho' = ||r||^2 (FP64 across the CTA, fixed-order last-CTA sum);
// for active shifts first the shifted direction of this iteration,
// p_s = zeta_k r + b_s p_s (r before its update: the direction kernel of the
// previous iteration left it to this pass, which reads r anyway), then
// x_s += a_s p_s.  Each lane owns CPL consecutive columns of a row (16-byte
// vector accesses); a shift's x_s and p_s are touched only by lanes that
// have an active column for it.
template <typename T, int KS>
__global__ void __launch_bounds__(VNE_THREADS, 2) k_cg_update(CgVectors<T> v, CgState st) {
    constexpr int CPL = LaneVec<T>::CPL;
    constexpr int LPR = KS / CPL;            // lanes per row
    constexpr int RPI = VNE_THREADS / LPR;   // rows per iteration
    const int panel = blockIdx.x / v.tiles_per_panel, tile = blockIdx.x % v.tiles_per_panel;
    const RowTile t = v.tiles[tile];
    const int sub = threadIdx.x % LPR, rs = threadIdx.x / LPR;
    const int cofs = sub * CPL;
    const size_t pofs = (size_t)panel * v.n * KS;
    // per-column coefficients in shared memory; this lane's active columns
    // as a bit mask (bit s * CPL + q)
    __shared__ __align__(16) T s_as[kMaxShifts][KS], s_z[kMaxShifts][KS], s_b[kMaxShifts][KS];
    for (int i = threadIdx.x; i < kMaxShifts * KS; i += VNE_THREADS) {
        const int sh = i / KS, cc = i % KS;
        const size_t o = (size_t)sh * st.K + panel * KS + cc;
        const bool on = sh < st.nshift && st.active[o];
        s_as[sh][cc] = on ? (T)st.as[o] : (T)0;
        s_z[sh][cc] = on ? (T)st.zeta[o] : (T)0;  // zeta_k
        s_b[sh][cc] = on ? (T)st.bs[o] : (T)0;    // b_s of the previous iteration
    }
    uint32_t amask = 0;
#pragma unroll
    for (int sh = 0; sh < kMaxShifts; sh++)
#pragma unroll
        for (int q = 0; q < CPL; q++)
            if (sh < st.nshift && st.active[(size_t)sh * st.K + panel * KS + cofs + q]) amask |= 1u << (sh * CPL + q);
    __syncthreads();
    T a[CPL];
#pragma unroll
    for (int q = 0; q < CPL; q++) a[q] = (T)st.a[panel * KS + cofs + q];
    T* R = v.r + pofs;
    const T* Q = v.q + pofs;
    double acc[CPL];
    T accf[CPL];
#pragma unroll
    for (int q = 0; q < CPL; q++) {
        acc[q] = 0.0;
        accf[q] = (T)0;
    }
    int cnt = 0;
    for (int r = t.row_begin + rs; r < t.row_end; r += RPI) {
        const size_t o = (size_t)r * KS + cofs;
        // every load of the row first (the pointers may alias as far as the
        // compiler knows, so a store between them would serialise them)
        T rv[CPL], qv[CPL];
        load_lane(R + o, rv);
        load_lane_stream(Q + o, qv);
        T xv[kMaxShifts][CPL], pv[kMaxShifts][CPL];
#pragma unroll
        for (int sh = 0; sh < kMaxShifts; sh++)
            if ((amask >> (sh * CPL)) & ((1u << CPL) - 1u)) {
                load_lane(v.x[sh] + pofs + o, xv[sh]);
                load_lane_stream(v.ps[sh] + pofs + o, pv[sh]);
            }
        T r0[CPL];  // r_k, for the shifted directions
#pragma unroll
        for (int q = 0; q < CPL; q++) {
            r0[q] = rv[q];
            rv[q] -= a[q] * qv[q];
            accf[q] += rv[q] * rv[q];
        }
        store_lane(R + o, rv);
        if (++cnt == 16) {
#pragma unroll
            for (int q = 0; q < CPL; q++) {
                acc[q] += (double)accf[q];
                accf[q] = (T)0;
            }
            cnt = 0;
        }
#pragma unroll
        for (int sh = 0; sh < kMaxShifts; sh++) {
            const uint32_t m = (amask >> (sh * CPL)) & ((1u << CPL) - 1u);
            if (!m) continue;
            T cv[CPL], zv[CPL], bv[CPL];
            load_lane(&s_as[sh][cofs], cv);
            load_lane(&s_z[sh][cofs], zv);
            load_lane(&s_b[sh][cofs], bv);
#pragma unroll
            for (int q = 0; q < CPL; q++)
                if (m & (1u << q)) {
                    pv[sh][q] = zv[q] * r0[q] + bv[q] * pv[sh][q];
                    xv[sh][q] += cv[q] * pv[sh][q];
                }
            store_lane(v.ps[sh] + pofs + o, pv[sh]);
            store_lane(v.x[sh] + pofs + o, xv[sh]);
        }
    }
    __shared__ double red[RPI][KS];
#pragma unroll
    for (int q = 0; q < CPL; q++) red[rs][cofs + q] = acc[q] + (double)accf[q];
    __syncthreads();
    if (threadIdx.x < KS) {
        double sum = 0.0;
        for (int q = 0; q < RPI; q++) sum += red[q][threadIdx.x];
        v.part[((size_t)panel * v.tiles_per_panel + tile) * KS + threadIdx.x] = sum;
    }
    // last CTA of the panel sums the partials in tile order
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(v.counter + panel, 1u) == (unsigned)(v.tiles_per_panel - 1));
    __syncthreads();
    if (s_last) {
        __threadfence();
        if (threadIdx.x < KS) {
            double sum = 0.0;
            for (int i = 0; i < v.tiles_per_panel; i++)
                sum += __ldcg(&v.part[((size_t)panel * v.tiles_per_panel + i) * KS + threadIdx.x]);
            st.rho_new[panel * KS + threadIdx.x] = sum;
        }
        if (threadIdx.x == 0) v.counter[panel] = 0u;
    }
}

// p = r + b p (the shifted directions are formed by the next k_cg_update)
template <typename T, int KS>
__global__ void __launch_bounds__(VNE_THREADS) k_cg_direction(CgVectors<T> v, CgState st) {
    constexpr int CPL = LaneVec<T>::CPL;
    constexpr int LPR = KS / CPL;
    constexpr int RPI = VNE_THREADS / LPR;
    const int panel = blockIdx.x / v.tiles_per_panel, tile = blockIdx.x % v.tiles_per_panel;
    const RowTile t = v.tiles[tile];
    const int sub = threadIdx.x % LPR, rs = threadIdx.x / LPR;
    const int cofs = sub * CPL;
    const size_t pofs = (size_t)panel * v.n * KS;
    T b[CPL];
#pragma unroll
    for (int q = 0; q < CPL; q++) b[q] = (T)st.b[panel * KS + cofs + q];
    const T* R = v.r + pofs;
    T* Pp = v.p + pofs;
    for (int r = t.row_begin + rs; r < t.row_end; r += RPI) {
        const size_t o = (size_t)r * KS + cofs;
        T rv[CPL], pv[CPL];
        load_lane_stream(R + o, rv);
        load_lane(Pp + o, pv);
#pragma unroll
        for (int q = 0; q < CPL; q++) pv[q] = rv[q] + b[q] * pv[q];
        store_lane(Pp + o, pv);
    }
}

// Per-column Cholesky of the column-scaled Gram matrix in pole order.  A
// column whose pivot (squared relative remainder) is <= drop is dependent on
// the kept ones and is dropped.  Returns the kept count; R (upper, kept
// columns) and D (column scales) are outputs.
__device__ int gram_cholesky(const double* Mg, int nb, int K, int c, double drop, double (&R)[kMaxBasis][kMaxBasis],
                             double (&D)[kMaxBasis], int (&keep)[kMaxBasis]) {
    for (int a = 0; a < nb; a++) {
        double maa = Mg[((size_t)a * nb + a) * K + c];
        D[a] = maa > 0.0 ? 1.0 / sqrt(maa) : 0.0;
    }
    int r = 0;
    for (int a = 0; a < nb; a++) {
        if (D[a] == 0.0) continue;
        double col[kMaxBasis];
        double s = 1.0;
        for (int i = 0; i < r; i++) {
            double v = Mg[((size_t)keep[i] * nb + a) * K + c] * D[keep[i]] * D[a];
            for (int l = 0; l < i; l++) v -= R[l][i] * col[l];
            col[i] = v / R[i][i];
            s -= col[i] * col[i];
        }
        if (s <= drop) continue;
        for (int i = 0; i < r; i++) R[i][r] = col[i];
        R[r][r] = sqrt(s);
        keep[r++] = a;
    }
    return r;
}

// Pass 1: X[c] = P D R^{-1} (nb x nb, rows by original column, zero for
// dropped ones) so that W X has orthonormal columns up to rounding; the
// second pass re-orthonormalises W X from its own Gram matrix (Cholesky-QR2).
__global__ void k_rational_pass1(const double* Mg, int nb, int K, double drop, double* X) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= K) return;
    double R[kMaxBasis][kMaxBasis], D[kMaxBasis];
    int keep[kMaxBasis];
    const int r = gram_cholesky(Mg, nb, K, c, drop, R, D, keep);
    for (int i = 0; i < nb * nb; i++) X[(size_t)i * K + c] = 0.0;
    for (int j = 0; j < r; j++) {
        // column j of R^{-1} (back substitution)
        double x[kMaxBasis];
        x[j] = 1.0 / R[j][j];
        for (int i = j - 1; i >= 0; i--) {
            double v = 0.0;
            for (int l = i + 1; l <= j; l++) v += R[i][l] * x[l];
            x[i] = -v / R[i][i];
        }
        for (int i = 0; i <= j; i++) X[((size_t)keep[i] * nb + j) * K + c] = D[keep[i]] * x[i];
    }
}

// Pass 2: orthonormalise the transformed basis, project A, diagonalise by
// cyclic Jacobi, psi = ||c||^2 sum_k z_{1k}^2 f(mu_k).  c2 = ||c||^2.
__global__ void k_rational_pass2(const double* Mg, const double* Kg, const double* c2v, int nb, int K, double drop,
                                 double* psi, int* rank_out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= K) return;
    const double c2 = c2v[(size_t)0 * K + c];
    double R[kMaxBasis][kMaxBasis], D[kMaxBasis];
    int keep[kMaxBasis];
    if (!(c2 > 0.0)) {
        psi[c] = 0.0;
        rank_out[c] = 0;
        return;
    }
    const int r = gram_cholesky(Mg, nb, K, c, drop, R, D, keep);
    double Ri[kMaxBasis][kMaxBasis];
    for (int j = 0; j < r; j++) {
        for (int i = 0; i < r; i++) Ri[i][j] = 0.0;
        Ri[j][j] = 1.0 / R[j][j];
        for (int i = j - 1; i >= 0; i--) {
            double v = 0.0;
            for (int l = i + 1; l <= j; l++) v += R[i][l] * Ri[l][j];
            Ri[i][j] = -v / R[i][i];
        }
    }
    // A_m = Ri^T Kt Ri with Kt the scaled, symmetrised W^T A W on kept columns
    double T1[kMaxBasis][kMaxBasis], Am[kMaxBasis][kMaxBasis];
    for (int i = 0; i < r; i++)
        for (int j = 0; j < r; j++) {
            double v = 0.0;
            for (int l = 0; l <= j; l++) {
                const int a = keep[i], b = keep[l];
                const double kab = 0.5 * (Kg[((size_t)a * nb + b) * K + c] + Kg[((size_t)b * nb + a) * K + c]);
                v += kab * D[a] * D[b] * Ri[l][j];
            }
            T1[i][j] = v;
        }
    for (int i = 0; i < r; i++)
        for (int j = 0; j < r; j++) {
            double v = 0.0;
            for (int l = 0; l <= i; l++) v += Ri[l][i] * T1[l][j];
            Am[i][j] = v;
        }
    double Z[kMaxBasis][kMaxBasis];
    for (int i = 0; i < r; i++)
        for (int j = 0; j < r; j++) Z[i][j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 30; sweep++) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < r; i++)
            for (int j = 0; j < r; j++) {
                tot += Am[i][j] * Am[i][j];
                if (i != j) off += Am[i][j] * Am[i][j];
            }
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < r; p++)
            for (int q = p + 1; q < r; q++) {
                double apq = Am[p][q];
                if (apq == 0.0) continue;
                double theta = (Am[q][q] - Am[p][p]) / (2.0 * apq);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
                for (int k = 0; k < r; k++) {
                    double akp = Am[k][p], akq = Am[k][q];
                    Am[k][p] = cs * akp - sn * akq;
                    Am[k][q] = sn * akp + cs * akq;
                }
                for (int k = 0; k < r; k++) {
                    double apk = Am[p][k], aqk = Am[q][k];
                    Am[p][k] = cs * apk - sn * aqk;
                    Am[q][k] = sn * apk + cs * aqk;
                }
                for (int k = 0; k < r; k++) {
                    double zkp = Z[k][p], zkq = Z[k][q];
                    Z[k][p] = cs * zkp - sn * zkq;
                    Z[k][q] = sn * zkp + cs * zkq;
                }
            }
    }
    double s = 0.0;
    for (int k = 0; k < r; k++) s += Z[0][k] * Z[0][k] * f_ent(Am[k][k]);
    psi[c] = c2 * s;
    rank_out[c] = r;
}

template <typename T, int KS>
__global__ void __launch_bounds__(VNE_THREADS) k_cgs_scale(T* v, const double* orig2, const double* rem2,
                                                           double drop2, int n, int K, int tiles_per_panel,
                                                           const RowTile* tiles) {
    const int panel = blockIdx.x / tiles_per_panel, tile = blockIdx.x % tiles_per_panel;
    const RowTile t = tiles[tile];
    const int c = threadIdx.x % KS, rsub = threadIdx.x / KS;
    constexpr int RPI = VNE_THREADS / KS;
    const int col = panel * KS + c;
    const double r2 = rem2[col];
    const double s = (r2 > 0.0 && r2 > drop2 * orig2[col]) ? 1.0 / sqrt(r2) : 0.0;
    T* V = v + (size_t)panel * n * KS;
    for (int r = t.row_begin + rsub; r < t.row_end; r += RPI) V[(size_t)r * KS + c] = (T)(s * (double)V[(size_t)r * KS + c]);
}

template <typename T>
cudaError_t launch_cgs_scale(T* v, const double* orig2, const double* rem2, double drop, int n, int K, int ks,
                             int tiles_per_panel, const RowTile* tiles, cudaStream_t st) {
    dim3 grid((K / ks) * tiles_per_panel);
    const double d2 = drop * drop;
    if (ks == 4) k_cgs_scale<T, 4><<<grid, VNE_THREADS, 0, st>>>(v, orig2, rem2, d2, n, K, tiles_per_panel, tiles);
    else if (ks == 8) k_cgs_scale<T, 8><<<grid, VNE_THREADS, 0, st>>>(v, orig2, rem2, d2, n, K, tiles_per_panel, tiles);
    else if (ks == 16) k_cgs_scale<T, 16><<<grid, VNE_THREADS, 0, st>>>(v, orig2, rem2, d2, n, K, tiles_per_panel, tiles);
    else if (ks == 32) k_cgs_scale<T, 32><<<grid, VNE_THREADS, 0, st>>>(v, orig2, rem2, d2, n, K, tiles_per_panel, tiles);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}
template cudaError_t launch_cgs_scale<float>(float*, const double*, const double*, double, int, int, int, int,
                                             const RowTile*, cudaStream_t);
template cudaError_t launch_cgs_scale<double>(double*, const double*, const double*, double, int, int, int, int,
                                              const RowTile*, cudaStream_t);

// Per-column basis change: out_j = sum_i in_i X[i][j] (X per column, FP64,
// staged in shared memory in the data precision).
template <typename T, int KS>
__global__ void __launch_bounds__(VNE_THREADS) k_block_transform(BlockTransform<T> bt) {
    constexpr int RPI = VNE_THREADS / KS;
    const int panel = blockIdx.x / bt.tiles_per_panel, tile = blockIdx.x % bt.tiles_per_panel;
    const RowTile t = bt.tiles[tile];
    const int c = threadIdx.x % KS, rs = threadIdx.x / KS;
    const int col = panel * KS + c;
    extern __shared__ __align__(16) unsigned char bt_smem[];
    T(*sx)[KS] = reinterpret_cast<T(*)[KS]>(bt_smem);  // [nb * nb][KS]
    for (int idx = threadIdx.x; idx < bt.nb * bt.nb * KS; idx += VNE_THREADS) {
        const int e = idx / KS, cc = idx % KS;
        sx[e][cc] = (T)bt.X[(size_t)e * bt.K + panel * KS + cc];
    }
    __syncthreads();
    const size_t pofs = (size_t)panel * bt.n * KS;
    for (int r = t.row_begin + rs; r < t.row_end; r += RPI) {
        const size_t o = pofs + (size_t)r * KS + c;
        T v[kMaxBasis];
        for (int i = 0; i < bt.nb; i++) v[i] = bt.in[i][o];
        for (int j = 0; j < bt.nb; j++) {
            T acc = (T)0;
            for (int i = 0; i < bt.nb; i++) acc += v[i] * sx[i * bt.nb + j][c];
            bt.out[j][o] = acc;
        }
    }
    (void)col;
}

// ---------------------------------------------------------------------------
// Gram matrices W^T W and W^T (A W) per column in one pass over the vectors
// (a kernel per pair of vectors would read every vector about nb times).  A
// CTA takes a range of rows of one panel in tiles of kGramRows rows: all 2 nb
// vectors' tile rows go to shared memory, and each thread accumulates a
// fixed set of (pair, column) outputs; the outputs are split into groups of
// kGramOut so that a thread holds at most kGramPer of them.  Sums per tile in
// the data precision (16 rows, as the pairwise kernel), FP64 across tiles,
// FP64 fixed-order sum over the row ranges.
constexpr int kGramRows = 16;
constexpr int kGramPer = 16;
constexpr int kGramOut = VNE_THREADS * kGramPer;

template <typename T, int KS>
__global__ void __launch_bounds__(VNE_THREADS) k_multi_gram(MultiGram<T> g) {
    extern __shared__ __align__(16) unsigned char mg_smem[];
    T* sv = reinterpret_cast<T*>(mg_smem);  // [2 nb][kGramRows][KS]
    __shared__ unsigned char s_x[kGramOut / KS + 1], s_y[kGramOut / KS + 1];
    const int chunk = blockIdx.x, grp = blockIdx.y, panel = blockIdx.z;
    const int nb = g.nb, nu = nb * (nb + 1) / 2, npair = 2 * nu;
    const int o_begin = grp * kGramOut, o_end = min(npair * KS, o_begin + kGramOut);
    // pair -> (x vector, y vector) for this group's pairs; y >= nb is AW
    const int p_begin = o_begin / KS, p_end = (o_end + KS - 1) / KS;
    for (int pr = p_begin + threadIdx.x; pr < p_end; pr += VNE_THREADS) {
        const int half = pr >= nu, q = half ? pr - nu : pr;
        int a = 0, rem = q;
        while (rem >= nb - a) {
            rem -= nb - a;
            a++;
        }
        s_x[pr - p_begin] = (unsigned char)a;
        s_y[pr - p_begin] = (unsigned char)(a + rem + (half ? nb : 0));
    }
    const int rows_per = (g.n + g.chunks - 1) / g.chunks;
    const int r_begin = chunk * rows_per, r_end = min(g.n, r_begin + rows_per);
    const size_t pofs = (size_t)panel * g.n * KS;
    double acc[kGramPer];
#pragma unroll
    for (int j = 0; j < kGramPer; j++) acc[j] = 0.0;
    const int nvec = 2 * nb;
    for (int r0 = r_begin; r0 < r_end; r0 += kGramRows) {
        const int rows = min(kGramRows, r_end - r0);
        __syncthreads();
        for (int idx = threadIdx.x; idx < nvec * kGramRows * KS; idx += VNE_THREADS) {
            const int v = idx / (kGramRows * KS), e = idx % (kGramRows * KS), rr = e / KS;
            const T* src = v < nb ? g.w[v] : g.aw[v - nb];
            sv[idx] = rr < rows ? src[pofs + (size_t)(r0 + rr) * KS + (e % KS)] : (T)0;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kGramPer; j++) {
            const int o = o_begin + threadIdx.x + j * VNE_THREADS;
            if (o >= o_end) break;
            const int pr = o / KS, c = o % KS;
            const T* X = sv + (size_t)s_x[pr - p_begin] * kGramRows * KS + c;
            const T* Y = sv + (size_t)s_y[pr - p_begin] * kGramRows * KS + c;
            T t = (T)0;
#pragma unroll
            for (int rr = 0; rr < kGramRows; rr++) t += X[rr * KS] * Y[rr * KS];
            acc[j] += (double)t;
        }
    }
    const size_t gbase = (((size_t)panel * g.groups + grp) * g.chunks + chunk) * kGramOut;
#pragma unroll
    for (int j = 0; j < kGramPer; j++) {
        const int o = o_begin + threadIdx.x + j * VNE_THREADS;
        if (o < o_end) g.part[gbase + (o - o_begin)] = acc[j];
    }
}

// out[pair][panel * KS + c] = fixed-order sum over the row ranges
__global__ void k_multi_gram_reduce(const double* part, int panels, int groups, int chunks, int ks, int npair,
                                    double* out) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const int K = panels * ks;
    if (idx >= npair * K) return;
    const int pr = idx / K, col = idx % K, panel = col / ks, c = col % ks;
    const int o = pr * ks + c, grp = o / kGramOut, oo = o % kGramOut;
    double s = 0.0;
    for (int ch = 0; ch < chunks; ch++) s += part[(((size_t)panel * groups + grp) * chunks + ch) * kGramOut + oo];
    out[(size_t)pr * K + col] = s;
}

// Lanczos tridiagonal of A from the seed CG's scalars (the CG-Lanczos
// relation): with step lengths a_i and direction coefficients b_i of CG on
// A + s0 I, T_{i+1,i+1} = 1/a_i + b_{i-1}/a_{i-1} - s0 (no second term at
// i = 0) and T_{i+1,i+2} = sqrt(b_i)/a_i.  An off-diagonal at or below tau
// (the Lanczos breakdown threshold) is set to 0: the Krylov space is
// invariant there, and the rows after it are not used.  History rows
// [i][K], i < k.
__global__ void k_cg_tridiag(const double* ah, const double* bh, int K, int k, double s0, double tau,
                             double* diag, double* off) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= K) return;
    double prev = 0.0;  // b_{i-1} / a_{i-1}
    for (int i = 0; i < k; i++) {
        const double a = ah[(size_t)i * K + c], b = bh[(size_t)i * K + c];
        const double t = sqrt(b) / a;
        diag[(size_t)i * K + c] = 1.0 / a + prev - s0;
        off[(size_t)i * K + c] = t > tau ? t : 0.0;
        prev = b / a;
    }
}

// Full [nb][nb][K] Gram layout from its upper triangle, pairs (a <= b)
// numbered row by row.
__global__ void k_gram_mirror(const double* uniq, int nb, int K, double* full) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)nb * nb * K) return;
    const int c = (int)(idx % K), b = (int)((idx / K) % nb), a = (int)(idx / ((size_t)K * nb));
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    const size_t pr = (size_t)lo * nb - (size_t)lo * (lo - 1) / 2 + (hi - lo);
    full[idx] = uniq[pr * K + c];
}

// ---------------------------------------------------------------------------

cudaError_t launch_cg_scalars_a(const CgState& st, cudaStream_t s) {
    k_cg_scalars_a<<<(st.K + 63) / 64, 64, 0, s>>>(st);
    return cudaGetLastError();
}
cudaError_t launch_cg_scalars_b(const CgState& st, cudaStream_t s) {
    k_cg_scalars_b<<<(st.K + 63) / 64, 64, 0, s>>>(st);
    return cudaGetLastError();
}

#define VNE_KS_SWITCH(T, ks, CALL)                                        \
    do {                                                                  \
        if ((ks) == 4) { constexpr int KS = 4; CALL; }                    \
        else if ((ks) == 8) { constexpr int KS = 8; CALL; }               \
        else if ((ks) == 16) { constexpr int KS = 16; CALL; }             \
        else if ((ks) == 32) { constexpr int KS = 32; CALL; }             \
        else return cudaErrorInvalidValue;                                \
    } while (0)

template <typename T>
cudaError_t launch_cg_update(const CgVectors<T>& v, const CgState& st, int ks, int panels, cudaStream_t s) {
    VNE_KS_SWITCH(T, ks, (k_cg_update<T, KS><<<panels * v.tiles_per_panel, VNE_THREADS, 0, s>>>(v, st)));
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_cg_direction(const CgVectors<T>& v, const CgState& st, int ks, int panels, cudaStream_t s) {
    VNE_KS_SWITCH(T, ks, (k_cg_direction<T, KS><<<panels * v.tiles_per_panel, VNE_THREADS, 0, s>>>(v, st)));
    return cudaGetLastError();
}
template <typename T, int KS>
cudaError_t multi_gram_ks(const MultiGram<T>& g, cudaStream_t s) {
    const size_t smem = (size_t)2 * g.nb * kGramRows * KS * sizeof(T);
    // the static pair tables (about 2 KB) count against the 48 KB default too
    if (smem + 4096 > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_multi_gram<T, KS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_multi_gram<T, KS><<<dim3(g.chunks, g.groups, g.panels), VNE_THREADS, smem, s>>>(g);
    return cudaSuccess;
}

template <typename T>
cudaError_t launch_multi_gram(MultiGram<T> g, double* out, cudaStream_t s) {
    if (g.nb < 1 || g.nb > 24) return cudaErrorInvalidValue;
    const int npair = g.nb * (g.nb + 1);
    g.groups = (npair * g.ks + kGramOut - 1) / kGramOut;
    cudaError_t e = cudaSuccess;
    VNE_KS_SWITCH(T, g.ks, (e = multi_gram_ks<T, KS>(g, s)));
    if (e != cudaSuccess) return e;
    const int K = g.panels * g.ks;
    k_multi_gram_reduce<<<(npair * K + 255) / 256, 256, 0, s>>>(g.part, g.panels, g.groups, g.chunks, g.ks, npair,
                                                                 out);
    return cudaGetLastError();
}
template cudaError_t launch_multi_gram<float>(MultiGram<float>, double*, cudaStream_t);
template cudaError_t launch_multi_gram<double>(MultiGram<double>, double*, cudaStream_t);

cudaError_t launch_cg_tridiag(const double* ah, const double* bh, int K, int k, double s0, double tau, double* diag,
                              double* off, cudaStream_t s) {
    if (k <= 0) return cudaSuccess;
    k_cg_tridiag<<<(K + 63) / 64, 64, 0, s>>>(ah, bh, K, k, s0, tau, diag, off);
    return cudaGetLastError();
}
cudaError_t launch_gram_mirror(const double* uniq, int nb, int K, double* full, cudaStream_t s) {
    const size_t total = (size_t)nb * nb * K;
    if (total == 0) return cudaSuccess;
    k_gram_mirror<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(uniq, nb, K, full);
    return cudaGetLastError();
}
cudaError_t launch_rational_pass1(const double* M, int nb, int K, double drop, double* X, cudaStream_t s) {
    if (nb > kMaxBasis) return cudaErrorInvalidValue;
    k_rational_pass1<<<(K + 31) / 32, 32, 0, s>>>(M, nb, K, drop, X);
    return cudaGetLastError();
}
cudaError_t launch_rational_pass2(const double* M, const double* Kmat, const double* c2, int nb, int K, double drop,
                                  double* psi, int* rank, cudaStream_t s) {
    if (nb > kMaxBasis) return cudaErrorInvalidValue;
    k_rational_pass2<<<(K + 31) / 32, 32, 0, s>>>(M, Kmat, c2, nb, K, drop, psi, rank);
    return cudaGetLastError();
}
// the basis-change matrix (nb^2 x KS values) lives in dynamic shared memory,
// beyond 48 KB for the largest bases
template <typename T, int KS>
cudaError_t block_transform_ks(const BlockTransform<T>& bt, int panels, size_t smem, cudaStream_t s) {
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_block_transform<T, KS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_block_transform<T, KS><<<panels * bt.tiles_per_panel, VNE_THREADS, smem, s>>>(bt);
    return cudaSuccess;
}

template <typename T>
cudaError_t launch_block_transform(const BlockTransform<T>& bt, int ks, int panels, cudaStream_t s) {
    if (bt.nb > kMaxBasis) return cudaErrorInvalidValue;
    const size_t smem = (size_t)bt.nb * bt.nb * ks * sizeof(T);
    cudaError_t e = cudaSuccess;
    VNE_KS_SWITCH(T, ks, (e = block_transform_ks<T, KS>(bt, panels, smem, s)));
    return e != cudaSuccess ? e : cudaGetLastError();
}

template cudaError_t launch_cg_update<float>(const CgVectors<float>&, const CgState&, int, int, cudaStream_t);
template cudaError_t launch_cg_update<double>(const CgVectors<double>&, const CgState&, int, int, cudaStream_t);
template cudaError_t launch_cg_direction<float>(const CgVectors<float>&, const CgState&, int, int, cudaStream_t);
template cudaError_t launch_cg_direction<double>(const CgVectors<double>&, const CgState&, int, int, cudaStream_t);
template cudaError_t launch_block_transform<float>(const BlockTransform<float>&, int, int, cudaStream_t);
template cudaError_t launch_block_transform<double>(const BlockTransform<double>&, int, int, cudaStream_t);

}  // namespace vne
