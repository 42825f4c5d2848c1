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

template <int MAXM>
__global__ void k_tridiag_quad(const double* __restrict__ alpha, const double* __restrict__ beta,
                               const double* __restrict__ norm2, const double* __restrict__ scale, int count,
                               int m, int ld, double* __restrict__ psi, int cols_per_cta) {
    if ((int)threadIdx.x >= cols_per_cta) return;
    int c = blockIdx.x * cols_per_cta + threadIdx.x;
    if (c >= count) return;
    double d[MAXM], e[MAXM], z[MAXM];
    int n = m;
    for (int j = 0; j < m; j++) {
        d[j] = alpha[(size_t)j * ld + c];
        z[j] = 0.0;
    }
    for (int j = 0; j + 1 < m; j++) {
        e[j] = beta[(size_t)j * ld + c];
        if (e[j] == 0.0) {
            n = j + 1;
            break;
        }
    }
    z[0] = 1.0;
    bool ok = symtri_qr_first_row(d, e, z, n);
    double sc = scale[c];
    double s = 0.0;
    for (int k = 0; k < n; k++) s += z[k] * z[k] * f_entropy(sc * d[k]);
    psi[c] = ok ? norm2[c] * s : nan("");
}

// warp per column; dynamic smem: Z [m][m] (row-major) per warp (1 warp / CTA).
// Every lane runs the scalar recurrence on its own copies (uniform control
// flow) and rotates the rows of Z it owns (rows lane, lane + 32, ...).
template <int R>
__global__ void k_tridiag_fvec(const double* __restrict__ alpha, const double* __restrict__ beta,
                               const double* __restrict__ scale, int count, int m, int ld,
                               double* __restrict__ zvec) {
    extern __shared__ double sm[];
    double* Z = sm;              // m*m
    double* d = sm + m * m;      // m
    double* e = d + m;           // m
    const int c = blockIdx.x;
    const int lane = threadIdx.x;
    if (c >= count) return;
    for (int idx = lane; idx < m * m; idx += 32) Z[idx] = ((idx / m) == (idx % m)) ? 1.0 : 0.0;
    for (int j = lane; j < m; j += 32) {
        d[j] = alpha[(size_t)j * ld + c];
        e[j] = (j + 1 < m) ? beta[(size_t)j * ld + c] : 0.0;
    }
    __syncwarp();
    int n = m;
    for (int j = 0; j + 1 < m; j++)
        if (e[j] == 0.0) {
            n = j + 1;
            break;
        }
    double dl[128], el[128];
    for (int j = 0; j < n; j++) {
        dl[j] = d[j];
        el[j] = e[j];
    }
    double* rows[R];
    int nr = 0;
    for (int q = 0; q < R; q++) {
        const int row = lane + 32 * q;
        rows[q] = Z + (size_t)(row < n ? row : 0) * m;
        if (row < n) nr = q + 1;
    }
    __syncwarp();
    bool ok = symtri_qr_rows<R>(dl, el, n, rows, nr);
    __syncwarp();
    double sc = scale[c];
    for (int row = lane; row < m; row += 32) {
        double acc = 0.0;
        if (row < n)
            for (int k = 0; k < n; k++) acc += Z[row * m + k] * f_entropy(sc * dl[k]) * Z[k];
        zvec[(size_t)row * ld + c] = ok ? acc : nan("");
    }
}

cudaError_t launch_tridiag_quad(const double* alpha, const double* beta, const double* norm2,
                                const double* scale_per_col, int count, int m, int ld, double* psi,
                                cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    // columns per CTA (one warp per CTA).  The FP64 pipe of an SM retires a
    // 32-lane FP64 instruction over many cycles, so the columns are spread
    // over all SMs first: ceil(count / SMs) columns per warp, at most 32.
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
    int cpw = (count + sms - 1) / sms;
    if (cpw > 32) cpw = 32;
    dim3 block(32), grid((count + cpw - 1) / cpw);
    if (m <= 32) k_tridiag_quad<32><<<grid, block, 0, st>>>(alpha, beta, norm2, scale_per_col, count, m, ld, psi, cpw);
    else if (m <= 64) k_tridiag_quad<64><<<grid, block, 0, st>>>(alpha, beta, norm2, scale_per_col, count, m, ld, psi, cpw);
    else if (m <= 128) k_tridiag_quad<128><<<grid, block, 0, st>>>(alpha, beta, norm2, scale_per_col, count, m, ld, psi, cpw);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_tridiag_fvec(const double* alpha, const double* beta, const double* scale_per_col, int count,
                                int m, int ld, double* zvec, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    if (m > 128) return cudaErrorInvalidValue;
    size_t smem = ((size_t)m * m + 2 * m) * sizeof(double);
    if (m <= 64) {
        cudaError_t e = cudaFuncSetAttribute(k_tridiag_fvec<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_tridiag_fvec<2><<<count, 32, smem, st>>>(alpha, beta, scale_per_col, count, m, ld, zvec);
    } else {
        cudaError_t e = cudaFuncSetAttribute(k_tridiag_fvec<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_tridiag_fvec<4><<<count, 32, smem, st>>>(alpha, beta, scale_per_col, count, m, ld, zvec);
    }
    return cudaGetLastError();
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

// Tensor-core Gram C = X^T Y for FP32 blocks (kx, ky <= 128): warp-level
// MMA m16n8k8 on TF32 operands with a three-product split (x = x_hi + x_lo,
// both TF32; x^T y ~ hi.hi + hi.lo + lo.hi), which keeps the products at
// FP32 accuracy.  The contraction reads each row of X and Y once (about 50
// flops per byte for 112 columns), so it is bound by HBM, not by the tensor
// pipe.  CTA: 8 warps in a 4 x 2 grid, each owning a 32 x 64 block of the
// 128 x 128 output; rows are streamed in 32-row slabs through padded shared
// memory; accumulation in FP32 over the CTA's rows, FP64 across CTAs.
__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <int KS>
__global__ void __launch_bounds__(256, 2) k_gram_tc(const float* __restrict__ X, int kx, const float* __restrict__ Y,
                                                    int ky, int n, int rows_per_chunk, double* __restrict__ part) {
    constexpr int LD = 136;  // padded row (128 + 8 floats): conflict-free fragment loads
    constexpr int SLAB = 32;
    constexpr int V_PER_ROW = KS / 4;  // float4 per row of one panel
    __shared__ __align__(16) float Xs[SLAB][LD];
    __shared__ __align__(16) float Ys[SLAB][LD];
    const int chunk = blockIdx.x;
    const int r_begin = chunk * rows_per_chunk;
    const int r_end = min(n, r_begin + rows_per_chunk);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = warp >> 1, wn = warp & 1;  // warp block: rows wm*32.., cols wn*64..
    const int g = lane >> 2, tq = lane & 3;
    const int px = kx / KS, py = ky / KS;     // panels of X and Y
    float acc[2][8][4];
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 8; j++)
#pragma unroll
            for (int q = 0; q < 4; q++) acc[i][j][q] = 0.f;
    // zero the columns no panel covers (they stay zero for the whole kernel)
    for (int idx = threadIdx.x; idx < SLAB * 128; idx += 256) {
        const int rl = idx >> 7, cl = idx & 127;
        if (cl >= kx) Xs[rl][cl] = 0.f;
        if (cl >= ky) Ys[rl][cl] = 0.f;
    }
    for (int rt = r_begin; rt < r_end; rt += SLAB) {
        // slab of SLAB rows: panel p of a block holds these rows contiguously
        // (SLAB * KS floats), so consecutive threads read consecutive float4s
        const int nx = px * SLAB * V_PER_ROW, ny = py * SLAB * V_PER_ROW;
        for (int idx = threadIdx.x; idx < nx + ny; idx += 256) {
            const bool isx = idx < nx;
            const int e = isx ? idx : idx - nx;
            const int p = e / (SLAB * V_PER_ROW), rem = e % (SLAB * V_PER_ROW);
            const int rl = rem / V_PER_ROW, c = (rem % V_PER_ROW) * 4;
            const int r = rt + rl;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (r < r_end) {
                const float* src = (isx ? X : Y) + (size_t)p * n * KS + (size_t)r * KS + c;
                v = __ldcs(reinterpret_cast<const float4*>(src));
            }
            float* dst = isx ? &Xs[rl][p * KS + c] : &Ys[rl][p * KS + c];
            *reinterpret_cast<float4*>(dst) = v;
        }
        __syncthreads();
#pragma unroll 1
        for (int k0 = 0; k0 < SLAB; k0 += 8) {
            // A = X^T (M = output rows, K = slab rows), two 16-row tiles per warp
            uint32_t ahi[2][4], alo[2][4];
#pragma unroll
            for (int i = 0; i < 2; i++) {
                const int m0 = wm * 32 + i * 16;
                const float vv[4] = {Xs[k0 + tq][m0 + g], Xs[k0 + tq][m0 + g + 8], Xs[k0 + tq + 4][m0 + g],
                                     Xs[k0 + tq + 4][m0 + g + 8]};
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    ahi[i][q] = to_tf32(vv[q]);
                    alo[i][q] = to_tf32(vv[q] - __uint_as_float(ahi[i][q]));
                }
            }
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const int n0 = wn * 64 + j * 8;
                const float w0 = Ys[k0 + tq][n0 + g], w1 = Ys[k0 + tq + 4][n0 + g];
                uint32_t bhi[2], blo[2];
                bhi[0] = to_tf32(w0);
                bhi[1] = to_tf32(w1);
                blo[0] = to_tf32(w0 - __uint_as_float(bhi[0]));
                blo[1] = to_tf32(w1 - __uint_as_float(bhi[1]));
#pragma unroll
                for (int i = 0; i < 2; i++) {
                    mma_tf32(acc[i][j], alo[i], bhi);
                    mma_tf32(acc[i][j], ahi[i], blo);
                    mma_tf32(acc[i][j], ahi[i], bhi);
                }
            }
        }
        __syncthreads();
    }
    // fragment (row g / g+8, col 2tq / 2tq+1) -> partial Gram of this chunk
#pragma unroll
    for (int i = 0; i < 2; i++)
#pragma unroll
        for (int j = 0; j < 8; j++)
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int row = wm * 32 + i * 16 + g + ((q & 2) ? 8 : 0);
                const int col = wn * 64 + j * 8 + 2 * tq + (q & 1);
                if (row < kx && col < ky) part[(size_t)chunk * kx * ky + (size_t)row * ky + col] = (double)acc[i][j][q];
            }
}

__global__ void k_gram_reduce(const double* __restrict__ part, int nchunks, int total, double* __restrict__ C) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    double s = 0.0;
    for (int c = 0; c < nchunks; c++) s += part[(size_t)c * total + idx];
    C[idx] = s;
}

template <typename T>
cudaError_t launch_gram(const T* X, int kx, const T* Y, int ky, int ks, int n, double* part, int nchunks, double* C,
                        cudaStream_t st) {
    if (kx <= 0 || ky <= 0) return cudaSuccess;
    if (sizeof(T) == 4 && kx <= 128 && ky <= 128) {
        // tensor-core path (FP32 data)
        int rpc = (n + nchunks - 1) / nchunks;
        rpc = ((rpc + 31) / 32) * 32;
        int chunks = rpc > 0 ? (n + rpc - 1) / rpc : 1;
        if (chunks < 1) chunks = 1;
        const float* Xf = reinterpret_cast<const float*>(X);
        const float* Yf = reinterpret_cast<const float*>(Y);
        if (ks == 8) k_gram_tc<8><<<chunks, 256, 0, st>>>(Xf, kx, Yf, ky, n, rpc, part);
        else if (ks == 16) k_gram_tc<16><<<chunks, 256, 0, st>>>(Xf, kx, Yf, ky, n, rpc, part);
        else if (ks == 32) k_gram_tc<32><<<chunks, 256, 0, st>>>(Xf, kx, Yf, ky, n, rpc, part);
        else return cudaErrorInvalidValue;
        int total = kx * ky;
        k_gram_reduce<<<(total + 255) / 256, 256, 0, st>>>(part, chunks, total, C);
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
                         double coef, cudaStream_t st) {
    if (kout > 128 || kin > 128) return cudaErrorInvalidValue;
    size_t smem = ((size_t)kin * 128 + 64 * (size_t)kin) * sizeof(T);
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int ntiles = (n + 63) / 64;
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
// Pivoted Cholesky G = P R^T R P^T (one CTA, FP64).  Stops when the largest
// remaining pivot is <= tol * max diag(G); rank r = pivots taken.  Writes
// Minv with Minv[piv[i]][c] = (R^{-1})[i][c] for i, c < r, zero elsewhere, so
// that Y Minv has orthonormal columns in exact arithmetic.
__global__ void k_chol_qr(const double* __restrict__ G, int k, double tol, double* __restrict__ Minv,
                          int* __restrict__ rank_out) {
    extern __shared__ double A[];  // k*k
    __shared__ int piv[128];
    __shared__ int s_p, s_rank;
    __shared__ double s_max0;
    for (int idx = threadIdx.x; idx < k * k; idx += blockDim.x) A[idx] = G[idx];
    for (int i = threadIdx.x; i < k; i += blockDim.x) piv[i] = i;
    __syncthreads();
    if (threadIdx.x == 0) {
        double mx = 0.0;
        for (int i = 0; i < k; i++) mx = fmax(mx, A[i * k + i]);
        s_max0 = mx;
        s_rank = k;
    }
    __syncthreads();
    for (int j = 0; j < k; j++) {
        if (threadIdx.x == 0) {
            int p = j;
            double best = A[j * k + j];
            for (int i = j + 1; i < k; i++)
                if (A[i * k + i] > best) {
                    best = A[i * k + i];
                    p = i;
                }
            s_p = (best > tol * s_max0 && best > 0.0) ? p : -1;
            if (s_p < 0) s_rank = j;
        }
        __syncthreads();
        const int p = s_p;
        if (p < 0) break;
        if (p != j) {
            for (int i = threadIdx.x; i < k; i += blockDim.x) {  // swap rows
                double t = A[j * k + i];
                A[j * k + i] = A[p * k + i];
                A[p * k + i] = t;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < k; i += blockDim.x) {  // swap columns
                double t = A[i * k + j];
                A[i * k + j] = A[i * k + p];
                A[i * k + p] = t;
            }
            if (threadIdx.x == 0) {
                int t = piv[j];
                piv[j] = piv[p];
                piv[p] = t;
            }
            __syncthreads();
        }
        const double rjj = sqrt(A[j * k + j]);
        __syncthreads();
        for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x) A[j * k + i] /= rjj;
        if (threadIdx.x == 0) A[j * k + j] = rjj;
        __syncthreads();
        const int rem = k - j - 1;
        for (int idx = threadIdx.x; idx < rem * rem; idx += blockDim.x) {
            int a = j + 1 + idx / rem, b = j + 1 + idx % rem;
            A[a * k + b] -= A[j * k + a] * A[j * k + b];
        }
        __syncthreads();
    }
    __syncthreads();
    const int r = s_rank;
    for (int idx = threadIdx.x; idx < k * k; idx += blockDim.x) Minv[idx] = 0.0;
    __syncthreads();
    // R^{-1} column by column (back substitution), one thread per column
    for (int c = threadIdx.x; c < r; c += blockDim.x) {
        double x[128];
        x[c] = 1.0 / A[c * k + c];
        for (int i = c - 1; i >= 0; i--) {
            double s = 0.0;
            for (int l = i + 1; l <= c; l++) s += A[i * k + l] * x[l];
            x[i] = -s / A[i * k + i];
        }
        for (int i = 0; i <= c; i++) Minv[(size_t)piv[i] * k + c] = x[i];
    }
    if (threadIdx.x == 0) *rank_out = r;
}

cudaError_t launch_chol_qr_factor(const double* G, int k, double tol, double* Minv, int* rank, cudaStream_t st) {
    if (k > 128 || k <= 0) return cudaErrorInvalidValue;
    size_t smem = (size_t)k * k * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_chol_qr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_chol_qr<<<1, 256, smem, st>>>(G, k, tol, Minv, rank);
    return cudaGetLastError();
}

template cudaError_t launch_gram<float>(const float*, int, const float*, int, int, int, double*, int, double*, cudaStream_t);
template cudaError_t launch_gram<double>(const double*, int, const double*, int, int, int, double*, int, double*, cudaStream_t);
template cudaError_t launch_apply<float>(const float*, int, const double*, int, const float*, float*, int, int, double, cudaStream_t);
template cudaError_t launch_apply<double>(const double*, int, const double*, int, const double*, double*, int, int, double, cudaStream_t);

}  // namespace vne
