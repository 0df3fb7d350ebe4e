// FP64 arithmetic of the randomized sketches (Algorithm 1/2): the Gram
// matrices of sketch blocks, the thin QR of the complex64 sketches by
// shifted Cholesky QR, and the Hermitian eigen-decomposition of the small
// Gram matrix that truncates Q Yt^H to rank r.  The tall factors (Y, Q, Yt)
// stay in the working precision; every k x k matrix derived from them
// (k <= 64 columns) is formed and factored with FP64 accuracy.
//
// FP64 on this GPU runs at 1/62 of the FP32 rate (1.25 against 78 TFLOP/s,
// measured) and its dependent chains are slow, so long serial FP64 code is
// avoided: the Gram of a complex64 block is accumulated with
// error-free transformations in FP32 arithmetic: every product a*b is split
// exactly into p + e (p = fl(a b), e = fma(a, b, -p)) and summed with
// TwoSum, which is Dot2 of Ogita, Rump and Oishi (SIAM J. Sci. Comput. 26,
// 2005): over a tile of 32 rows the result is as accurate as a sum in twice
// the working precision; tiles and row chunks are then added in FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cfloat>
#include <cmath>

#include "lsw_internal.cuh"

namespace lsw {

namespace {

constexpr int GT_ROWS = 32;   // rows per tile (one compensated sum)
constexpr int GT_MAXQ = 9;    // pairs per thread: 256 * 9 >= 64 * 65 / 2

// Row chunks per block for the Gram and the product kernels: down to one
// tile of 32 rows per CTA, about 1216 CTAs (8 per SM) over the batch, so
// that a few small blocks (the recompressions on the inversion's critical
// path) still spread over the GPU.
int sketch_chunks(int m, int batch) {
    return std::max(1, std::min((m + GT_ROWS - 1) / GT_ROWS, std::max(1, 1216 / batch)));
}

int grid_small(long long n, int bs = 256) {
    long long g = (n + bs - 1) / bs;
    return (int)std::max<long long>(1, std::min<long long>(g, 152LL * 32));
}

// ------------------------------------------------------ compensated Gram
// s + c accumulates a * b: p + e = a * b exactly, (s, q) = TwoSum(s, p),
// c += q + e.  The round-to-nearest intrinsics keep the compiler from
// contracting a product into a neighbouring add.
__device__ __forceinline__ void dot2(float a, float b, float& s, float& c) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    const float t = __fadd_rn(s, p);
    const float z = __fsub_rn(t, s);
    const float q = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
    s = t;
    c = __fadd_rn(c, __fadd_rn(q, e));
}

// upper-triangle pair index p -> (i, j), i <= j, p = j (j + 1) / 2 + i
__device__ __forceinline__ void tri_pair(int p, int& i, int& j) {
    int jj = (int)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);
    while ((jj + 1) * (jj + 2) / 2 <= p) ++jj;
    while (jj * (jj + 1) / 2 > p) --jj;
    j = jj;
    i = p - jj * (jj + 1) / 2;
}


// Partial Gram of rows [r0, r1) of block b: part[(b * nchunk + ch) * npair + p]
// for the upper-triangle pairs p.  Columns are staged in shared memory in
// tiles of 32 rows (odd stride: the lanes of a warp read different banks).
__global__ void __launch_bounds__(256)
k_gram_c64(const float2* __restrict__ Y, int m, int k, long long sY, int nchunk, double2* __restrict__ part,
           const int* __restrict__ active) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    float2* sy = reinterpret_cast<float2*>(sm_raw);   // k columns x (GT_ROWS + 1)
    const int b = blockIdx.y, ch = blockIdx.x;
    if (active && !active[b]) return;                 // this block needs no second pass
    const int rows_per = (m + nchunk - 1) / nchunk;
    const int r0 = ch * rows_per, r1 = min(m, r0 + rows_per);
    const float2* Yb = Y + (long long)b * sY;
    const int npair = k * (k + 1) / 2;
    int pi[GT_MAXQ], pj[GT_MAXQ];
    double2 acc[GT_MAXQ];
#pragma unroll
    for (int q = 0; q < GT_MAXQ; ++q) {
        const int p = threadIdx.x + q * 256;
        pi[q] = 0;
        pj[q] = 0;
        if (p < npair) tri_pair(p, pi[q], pj[q]);
        acc[q] = make_double2(0.0, 0.0);
    }
    for (int rr = r0; rr < r1; rr += GT_ROWS) {
        const int nr = min(GT_ROWS, r1 - rr);
        for (int e = threadIdx.x; e < GT_ROWS * k; e += 256) {
            const int c = e / GT_ROWS, r = e - c * GT_ROWS;
            sy[c * (GT_ROWS + 1) + r] = r < nr ? Yb[(long long)c * m + rr + r] : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < GT_MAXQ; ++q) {
            if (threadIdx.x + q * 256 < npair) {
                const float2* yi = sy + pi[q] * (GT_ROWS + 1);
                const float2* yj = sy + pj[q] * (GT_ROWS + 1);
                float sre = 0.f, cre = 0.f, sim = 0.f, cim = 0.f;
                for (int r = 0; r < nr; ++r) {
                    const float2 a = yi[r], v = yj[r];
                    // conj(a) * v = (ax vx + ay vy) + i (ax vy - ay vx)
                    dot2(a.x, v.x, sre, cre);
                    dot2(a.y, v.y, sre, cre);
                    dot2(a.x, v.y, sim, cim);
                    dot2(-a.y, v.x, sim, cim);
                }
                acc[q].x += (double)sre + (double)cre;
                acc[q].y += (double)sim + (double)cim;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < GT_MAXQ; ++q) {
        const int p = threadIdx.x + q * 256;
        if (p < npair) part[((long long)b * nchunk + ch) * npair + p] = acc[q];
    }
}

// G_b (k x k, full Hermitian, column-major) = sum over chunks, in FP64.
__global__ void k_gram_c64_reduce(const double2* __restrict__ part, int nchunk, int k, int batch, double2* G) {
    const int npair = k * (k + 1) / 2;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < batch * k * k; e += gridDim.x * blockDim.x) {
        const int b = e / (k * k), ij = e - b * k * k;
        const int j = ij / k, i = ij - j * k;
        const int lo = min(i, j), hi = max(i, j);
        const int p = hi * (hi + 1) / 2 + lo;
        // eight interleaved partial sums: short FP64 dependency chains
        double2 acc[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[u] = make_double2(0.0, 0.0);
        const double2* src = part + (long long)b * nchunk * npair + p;
        int c = 0;
        for (; c + 8 <= nchunk; c += 8) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const double2 v = src[(long long)(c + u) * npair];
                acc[u].x += v.x;
                acc[u].y += v.y;
            }
        }
        for (int u = 0; c < nchunk; ++c, ++u) {
            const double2 v = src[(long long)c * npair];
            acc[u].x += v.x;
            acc[u].y += v.y;
        }
        double2 s = make_double2(((acc[0].x + acc[1].x) + (acc[2].x + acc[3].x)) + ((acc[4].x + acc[5].x) + (acc[6].x + acc[7].x)),
                                 ((acc[0].y + acc[1].y) + (acc[2].y + acc[3].y)) + ((acc[4].y + acc[5].y) + (acc[6].y + acc[7].y)));
        if (i > j) s.y = -s.y;   // G(i, j) = conj(G(j, i))
        G[e] = s;
    }
}

// ------------------------------------------- Cholesky and R^-1 (FP64)
// One CTA per matrix: G + shift I = Lt D Lt^H (Lt unit lower triangular, D
// diagonal: the square-root-free Cholesky), then Xt = Lt^-1 and
// R^-1 = Xt^H D^-1/2 (R = D^1/2 Lt^H, so R^H R = G + shift I).
// Written for the rate and latency of FP64 on this GPU (2 FP64 lanes per
// cycle per SM): every multiply-add a thread issues is useful (the trailing
// triangle is enumerated through a table, not masked out of a square), a
// step waits on one barrier-separated phase of independent multiply-adds,
// the pivot's reciprocal (an FP32 estimate and two Newton steps, no FP64
// division) is formed by the thread that finishes the pivot while the
// others finish the step, and the square roots of D are taken once, at the
// end, for all columns at once.
// A non-positive pivot restarts the factorisation with a larger shift
// (1e-15 tr(G) / k, then x100, at most 12 times).  A block with tr(G) = 0
// gets Rinv = 0 (its Q is zero, which the truncation keeps as a zero block).
__device__ __forceinline__ double rsqrt64(double d) {
    float f = (float)d;
    double y = (f > 1e-37f && f < 1e37f) ? (double)rsqrtf(f) : 1.0 / sqrt(d);
    // y <- y (3 - d y^2) / 2, twice: relative error ~1e-7 -> ~1e-14 -> rounding
    for (int it = 0; it < 2; ++it) {
        const double e = fma(-d * y, y, 1.0);
        y = fma(0.5 * y, e, y);
    }
    return y;
}

__device__ __forceinline__ double rcp64(double d) {
    float f = (float)d;
    double y = (f > 1e-37f && f < 1e37f) ? (double)(1.0f / f) : 1.0 / d;
    // y <- y (2 - d y), twice
    for (int it = 0; it < 2; ++it) {
        const double e = fma(-d, y, 1.0);
        y = fma(y, e, y);
    }
    return y;
}

constexpr int CH_NT = 256;   // threads per matrix

template <typename C>
__global__ void __launch_bounds__(CH_NT)
k_chol_rinv(const double2* __restrict__ Gall, int k, int batch, double shift_rel, C* __restrict__ Rall,
            const int* __restrict__ active, int* __restrict__ need2) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int tid = threadIdx.x;
    const int mat = blockIdx.x;
    if (active && !active[mat]) return;
    const int ld = k + 1;
    // A: lower triangle = the matrix being factored (then Lt D), upper
    // triangle = U(j, l) = conj(Lt(l, j)), written as each column finishes
    double2* A = reinterpret_cast<double2*>(sm_raw);
    double2* X = A + (size_t)k * ld;                            // Xt = Lt^-1, lower
    double* dinv = reinterpret_cast<double*>(X + (size_t)k * ld);  // 1 / D(j)
    short2* tri = reinterpret_cast<short2*>(dinv + k);          // p -> (a, b), a <= b
    __shared__ double red[CH_NT / 32];
    __shared__ int fail;
    const double2* G = Gall + (long long)mat * k * k;
    C* Rout = Rall + (long long)mat * k * k;
    const int ntri = k * (k - 1) / 2;
    for (int p = tid; p < ntri; p += CH_NT) {
        int bb = (int)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);
        while ((bb + 1) * (bb + 2) / 2 <= p) ++bb;
        while (bb * (bb + 1) / 2 > p) --bb;
        tri[p] = make_short2((short)(p - bb * (bb + 1) / 2), (short)bb);
    }
    double tr = 0.0;
    for (int i = tid; i < k; i += CH_NT) tr += G[i * k + i].x;
    for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
    if ((tid & 31) == 0) red[tid >> 5] = tr;
    __syncthreads();
    tr = 0.0;
    for (int w = 0; w < CH_NT / 32; ++w) tr += red[w];
    tr /= k;
    if (!(tr > 0.0) || !isfinite(tr)) {
        const double fill = (tr == 0.0) ? 0.0 : NAN;
        for (int e = tid; e < k * k; e += CH_NT) { Rout[e].x = fill; Rout[e].y = fill; }
        if (need2 && tid == 0) need2[mat] = 0;
        return;
    }
    double shift = shift_rel * tr;
    const bool shifted0 = shift > 0.0;
    int attempts = 0;
    bool ok = false;
    for (int attempt = 0; attempt < 13 && !ok; ++attempt) {
        for (int e = tid; e < k * k; e += CH_NT) {
            const int j = e / k, i = e - j * k;
            if (i < j) continue;
            double2 v = G[e];
            if (i == j) { v.x += shift; v.y = 0.0; }
            A[j * ld + i] = v;
        }
        if (tid == 0) {
            const double d0 = G[0].x + shift;
            fail = (d0 > 0.0 && isfinite(d0)) ? 0 : 1;
            dinv[0] = rcp64(d0);
        }
        __syncthreads();
        for (int j = 0; j < k - 1 && !fail; ++j) {
            // column j of Lt, kept conjugated in row j: U(j, i) = conj(A(i, j)) / D(j)
            const double dj = dinv[j];
            for (int i = j + 1 + tid; i < k; i += CH_NT) {
                const double2 v = A[j * ld + i];
                A[i * ld + j] = make_double2(v.x * dj, -v.y * dj);
            }
            __syncthreads();
            // trailing triangle: A(i, l) -= A(i, j) U(j, l), j < l <= i; item
            // 0 (the next pivot) first, on thread 0, which then forms 1 / D(j+1)
            const int nt = k - 1 - j, T = nt * (nt + 1) / 2;
            for (int p = tid; p < T; p += CH_NT) {
                const short2 ab = tri[T - 1 - p];
                const int i = j + nt - ab.x, l = j + nt - ab.y;
                const double2 a = A[j * ld + i], u = A[l * ld + j];
                double2 v = A[l * ld + i];
                v.x = fma(-a.x, u.x, v.x);
                v.x = fma(a.y, u.y, v.x);
                v.y = fma(-a.x, u.y, v.y);
                v.y = fma(-a.y, u.x, v.y);
                A[l * ld + i] = v;
                if (p == 0) {
                    const double d = v.x;
                    if (!(d > 0.0) || !isfinite(d)) fail = 1;
                    dinv[j + 1] = rcp64(d);
                }
            }
            __syncthreads();
        }
        ok = fail == 0;
        __syncthreads();
        if (!ok) shift = shift > 0.0 ? shift * 100.0 : 1e-15 * tr;
        ++attempts;
    }
    if (!ok) {
        for (int e = tid; e < k * k; e += CH_NT) { Rout[e].x = NAN; Rout[e].y = NAN; }
        if (need2 && tid == 0) need2[mat] = 0;
        return;
    }
    // Xt = Lt^-1 in axpy form, every column at once: Xt starts as I; after
    // step t - 1 row t is final in every column c <= t, and step t removes it
    // from the rows below: Xt(i, c) -= Lt(i, t) Xt(t, c), Lt(i, t) = conj(U(t, i)).
    for (int e = tid; e < k * ld; e += CH_NT) {
        const int c = e / ld, i = e - c * ld;
        X[e] = make_double2(i == c ? 1.0 : 0.0, 0.0);
    }
    __syncthreads();
    for (int t = 0; t < k - 1; ++t) {
        const int nr = k - 1 - t, n = nr * (t + 1);
        const float rnr = 1.0f / (float)nr;
        for (int e = tid; e < n; e += CH_NT) {
            // e = c * nr + (i - t - 1); the float quotient is exact here
            // (e < 4096, nr < 64: the fraction is at least 1 / (2 nr) from an integer)
            const int c = (int)(((float)e + 0.5f) * rnr), i = t + 1 + (e - c * nr);
            const double2 u = A[i * ld + t], xt = X[c * ld + t];
            double2 v = X[c * ld + i];
            // v -= conj(u) xt
            v.x = fma(-u.x, xt.x, v.x);
            v.x = fma(-u.y, xt.y, v.x);
            v.y = fma(-u.x, xt.y, v.y);
            v.y = fma(u.y, xt.x, v.y);
            X[c * ld + i] = v;
        }
        __syncthreads();
    }
    // D^-1/2 for every column at once (reuses dinv)
    for (int j = tid; j < k; j += CH_NT) dinv[j] = rsqrt64(A[j * ld + j].x);
    __syncthreads();
    // Rinv(i, j) = conj(Xt(j, i)) D(j)^-1/2, upper triangular
    double fro = 0.0;
    for (int e = tid; e < k * k; e += CH_NT) {
        const int j = e / k, i = e - j * k;
        C v;
        if (i <= j) {
            const double2 xv = X[i * ld + j];
            const double s = dinv[j];
            v.x = xv.x * s;
            v.y = -xv.y * s;
            fro += (double)v.x * v.x + (double)v.y * v.y;
        } else {
            v.x = 0;
            v.y = 0;
        }
        Rout[e] = v;
    }
    if (need2) {
        // kappa_F = ||Y||_F ||R^-1||_F >= kappa_2(Y).  One pass of Cholesky QR
        // with an FP64-accurate Gram and product leaves Q^H Q - I ~ 1e-16
        // kappa^2: a second pass is needed above kappa ~ 1e3 (and after any
        // shift, which perturbs the factor on purpose).
        for (int o = 16; o > 0; o >>= 1) fro += __shfl_xor_sync(0xffffffffu, fro, o);
        __syncthreads();
        if ((tid & 31) == 0) red[tid >> 5] = fro;
        __syncthreads();
        if (tid == 0) {
            double rf = 0.0;
            for (int w = 0; w < CH_NT / 32; ++w) rf += red[w];
            const double kap2 = tr * k * rf;
            need2[mat] = (shifted0 || attempts > 0 || !(kap2 <= 1e6)) ? 1 : 0;
        }
    }
}

// Q = Y R^-1 in place, formed with FP64 accuracy in FP32 arithmetic: R^-1
// (FP64, upper triangular) is split into two FP32 parts, the products with
// the high part are summed by Dot2 and those with the low part are added to
// the compensation; the result is rounded to FP32 once.  Rows are
// independent, so each CTA loads a tile of rows into shared memory and
// writes its result over it.  Blocks whose active flag is 0 are skipped.
__global__ void __launch_bounds__(256)
k_rmul_dot2(float2* __restrict__ Y, int m, int k, long long sY, const double2* __restrict__ Rall,
            const int* __restrict__ active) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int b = blockIdx.y;
    if (active && !active[b]) return;
    float2* Rh = reinterpret_cast<float2*>(sm_raw);   // k x k
    float2* Rl = Rh + k * k;
    float2* yt = Rl + k * k;                           // k columns x (GT_ROWS + 1)
    const double2* R = Rall + (long long)b * k * k;
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
        const double2 v = R[e];
        const float hx = (float)v.x, hy = (float)v.y;
        Rh[e] = make_float2(hx, hy);
        Rl[e] = make_float2((float)(v.x - (double)hx), (float)(v.y - (double)hy));
    }
    float2* Yb = Y + (long long)b * sY;
    const int rows_per = (m + gridDim.x - 1) / gridDim.x;
    const int r0 = blockIdx.x * rows_per, r1 = min(m, r0 + rows_per);
    for (int rr = r0; rr < r1; rr += GT_ROWS) {
        const int nr = min(GT_ROWS, r1 - rr);
        __syncthreads();
        for (int e = threadIdx.x; e < GT_ROWS * k; e += blockDim.x) {
            const int c = e / GT_ROWS, r = e - c * GT_ROWS;
            yt[c * (GT_ROWS + 1) + r] = r < nr ? Yb[(long long)c * m + rr + r] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < GT_ROWS * k; e += blockDim.x) {
            const int j = e / GT_ROWS, r = e - j * GT_ROWS;
            if (r >= nr) continue;
            float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
            for (int t = 0; t <= j; ++t) {
                const float2 a = yt[t * (GT_ROWS + 1) + r], h = Rh[j * k + t], l = Rl[j * k + t];
                dot2(a.x, h.x, sr, cr);
                dot2(-a.y, h.y, sr, cr);
                dot2(a.x, h.y, si, ci);
                dot2(a.y, h.x, si, ci);
                cr = fmaf(a.x, l.x, fmaf(-a.y, l.y, cr));
                ci = fmaf(a.x, l.y, fmaf(a.y, l.x, ci));
            }
            Yb[(long long)j * m + rr + r] = make_float2(__fadd_rn(sr, cr), __fadd_rn(si, ci));
        }
    }
}

// ------------------------------- Rayleigh-Ritz projection (FP64 accuracy)
// B = V0^H G V0 for FP32 approximate eigenvectors V0 of the FP64 Hermitian G,
// formed with FP64 accuracy in FP32 arithmetic: G = Ghi + Glo (two FP32
// parts), W = G V0 by Dot2 over the Ghi terms with the Glo terms added to the
// compensation, kept as the pair Whi + Wlo; then B = V0^H (Whi + Wlo) the
// same way.  One CTA per matrix; B is written Hermitian (upper triangle
// computed, lower mirrored).  Small eigenvalues of G that FP32 could not
// separate inside G (below ~1e-7 of the largest) sit on B's diagonal with
// their own exponents, where an FP32 Jacobi resolves them.
__global__ void __launch_bounds__(1024)
k_rr_project(const double2* __restrict__ Gall, const float2* __restrict__ V0all, int k, double2* __restrict__ Ball) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int kk = k * k;
    float2* Ghi = reinterpret_cast<float2*>(sm_raw);
    float2* Glo = Ghi + kk;
    float2* V = Glo + kk;
    float2* Whi = V + kk;
    float2* Wlo = Whi + kk;
    const double2* G = Gall + (long long)blockIdx.x * kk;
    const float2* V0 = V0all + (long long)blockIdx.x * kk;
    double2* B = Ball + (long long)blockIdx.x * kk;
    for (int e = threadIdx.x; e < kk; e += blockDim.x) {
        const double2 g = G[e];
        const float hx = (float)g.x, hy = (float)g.y;
        Ghi[e] = make_float2(hx, hy);
        Glo[e] = make_float2((float)(g.x - (double)hx), (float)(g.y - (double)hy));
        V[e] = V0[e];
    }
    __syncthreads();
    // W(i, j) = sum_t G(i, t) V(t, j)
    for (int e = threadIdx.x; e < kk; e += blockDim.x) {
        const int j = e / k, i = e - j * k;
        float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
        for (int t = 0; t < k; ++t) {
            const float2 gh = Ghi[t * k + i], gl = Glo[t * k + i], v = V[j * k + t];
            dot2(gh.x, v.x, sr, cr);
            dot2(-gh.y, v.y, sr, cr);
            dot2(gh.x, v.y, si, ci);
            dot2(gh.y, v.x, si, ci);
            cr = fmaf(gl.x, v.x, fmaf(-gl.y, v.y, cr));
            ci = fmaf(gl.x, v.y, fmaf(gl.y, v.x, ci));
        }
        // renormalise the pair so that Whi carries the leading bits
        const float hr = __fadd_rn(sr, cr), hi = __fadd_rn(si, ci);
        Whi[e] = make_float2(hr, hi);
        Wlo[e] = make_float2(__fsub_rn(cr, __fsub_rn(hr, sr)), __fsub_rn(ci, __fsub_rn(hi, si)));
    }
    __syncthreads();
    // B(i, j) = sum_t conj(V(t, i)) W(t, j), i <= j
    const int npair = k * (k + 1) / 2;
    for (int p = threadIdx.x; p < npair; p += blockDim.x) {
        int i, j;
        tri_pair(p, i, j);
        float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
        for (int t = 0; t < k; ++t) {
            const float2 a = V[i * k + t], wh = Whi[j * k + t], wl = Wlo[j * k + t];
            // conj(a) * w = (ax wx + ay wy) + i (ax wy - ay wx)
            dot2(a.x, wh.x, sr, cr);
            dot2(a.y, wh.y, sr, cr);
            dot2(a.x, wh.y, si, ci);
            dot2(-a.y, wh.x, si, ci);
            cr = fmaf(a.x, wl.x, fmaf(a.y, wl.y, cr));
            ci = fmaf(a.x, wl.y, fmaf(-a.y, wl.x, ci));
        }
        const double br = (double)sr + (double)cr, bi = (double)si + (double)ci;
        if (i == j) {
            B[j * k + i] = make_double2(br, 0.0);
        } else {
            B[j * k + i] = make_double2(br, bi);
            B[i * k + j] = make_double2(br, -bi);
        }
    }
}

__global__ void k_up64(const float2* __restrict__ s, long long sS, double2* __restrict__ d, long long n, int batch) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n * batch; e += (long long)gridDim.x * blockDim.x) {
        const long long b = e / n, i = e - b * n;
        const float2 v = s[b * sS + i];
        d[e] = make_double2(v.x, v.y);
    }
}

__global__ void k_down32(const double2* __restrict__ s, float2* __restrict__ d, long long sD, long long n, int batch) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n * batch; e += (long long)gridDim.x * blockDim.x) {
        const long long b = e / n, i = e - b * n;
        const double2 v = s[e];
        d[b * sD + i] = make_float2((float)v.x, (float)v.y);
    }
}

}  // namespace

lsw_status gram64_c64(const float2* Y, int m, int k, long long sY, int batch, double2* G, cudaStream_t st,
                      const int* active) {
    if (batch <= 0 || k <= 0) return LSW_OK;
    if (k > 64) return LSW_ERR_INVALID_ARG;
    const int nchunk = sketch_chunks(m, batch);
    const int npair = k * (k + 1) / 2;
    DevBuf part;
    LSW_TRY(part.alloc(sizeof(double2) * (size_t)batch * nchunk * npair, st));
    KTimer kt("gram", st, 8.0 * batch * (double)m * k, 0.0);
    k_gram_c64<<<dim3(nchunk, batch), 256, sizeof(float2) * (GT_ROWS + 1) * k, st>>>(Y, m, k, sY, nchunk,
                                                                                        part.as<double2>(), active);
    LSW_LAUNCH_CHECK();
    k_gram_c64_reduce<<<grid_small((long long)batch * k * k), 256, 0, st>>>(part.as<double2>(), nchunk, k, batch, G);
    LSW_LAUNCH_CHECK();
    return LSW_OK;
}

template <typename R>
lsw_status chol_rinv(const double2* G, int k, int batch, double shift_rel, typename Cx<R>::T* Rinv, cudaStream_t st,
                     const int* active, int* need2) {
    typedef typename Cx<R>::T C;
    if (batch <= 0 || k <= 0) return LSW_OK;
    if (k > 64) return LSW_ERR_INVALID_ARG;
    const size_t per = sizeof(double2) * 2 * (size_t)k * (k + 1) + sizeof(double) * k +
                       sizeof(short2) * (size_t)(k * (k - 1) / 2 + 1);
    static std::atomic<bool> attr{false};
    if (!attr.load()) {
        LSW_CUDA(cudaFuncSetAttribute(k_chol_rinv<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        attr.store(true);
    }
    KTimer kt("chol", st, 0.0, 0.0);
    k_chol_rinv<C><<<batch, CH_NT, per, st>>>(G, k, batch, shift_rel, Rinv, active, need2);
    LSW_LAUNCH_CHECK();
    return LSW_OK;
}

lsw_status heev_c64(const double2* G, float2* V, int k, int batch, cudaStream_t st) {
    if (batch <= 0 || k <= 0) return LSW_OK;
    if (k > 64) return LSW_ERR_INVALID_ARG;
    // algorithmic work: the classical count of a Hermitian eigen-decomposition
    // with eigenvectors, 9 k^3 real flops for real symmetric, four times that
    // for complex (reads and writes of the k x k matrices only, in bytes)
    KTimer kt("heev", st, 24.0 * (double)k * k * batch, 36.0 * (double)k * k * k * batch);
    const size_t kk = (size_t)k * k;
    DevBuf V0, B, Z;
    LSW_TRY(V0.alloc(sizeof(float2) * kk * batch, st));
    LSW_TRY(B.alloc(sizeof(double2) * kk * batch, st));
    LSW_TRY(Z.alloc(sizeof(float2) * kk * batch, st));
    LSW_TRY(heev_jacobi<float>(G, V0.as<float2>(), k, batch, st, 2));
    static std::atomic<bool> attr{false};
    if (!attr.load()) {
        LSW_CUDA(cudaFuncSetAttribute(k_rr_project, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        attr.store(true);
    }
    // few matrices (the critical path of the recursive inversion): a CTA of
    // 1024 threads on each
    k_rr_project<<<batch, batch <= 2 * 152 ? 1024 : 128, sizeof(float2) * 5 * kk, st>>>(G, V0.as<float2>(), k,
                                                                                       B.as<double2>());
    LSW_LAUNCH_CHECK();
    LSW_TRY(heev_jacobi<float>(B.as<double2>(), Z.as<float2>(), k, batch, st, 1));
    const float2 one = make_float2(1.f, 0.f), zero = make_float2(0.f, 0.f);
    return gemm<float>('N', 'N', k, k, k, one, V0.as<float2>(), k, (long long)kk, Z.as<float2>(), k, (long long)kk,
                       zero, V, k, (long long)kk, batch, st);
}

// Thin QR of complex64 sketch blocks, Q returned in place of A (m x k, ld m,
// block stride sA).  Tall blocks (m >= 4k): Cholesky QR with FP64-accurate
// arithmetic in every step (Yamamoto, Nakatsukasa, Yanagisawa, Fukaya 2015,
// with the Gram and the product both accurate to ~1e-16): G = Y^H Y by
// Dot2, G + s I = R^H R in FP64 (s = 0, raised only on breakdown), Q = Y R^-1
// by Dot2 products in place.  Then Q^H Q - I ~ 1e-16 kappa(Y)^2 + u32, so a
// second identical pass on Q runs only for the blocks whose estimate
// kappa_F = ||Y||_F ||R^-1||_F exceeds 1e3 or whose factor needed a shift
// (a per-block flag on the device; the other blocks skip it).  Short blocks:
// Householder QR in FP64 on an upcast copy.
lsw_status qr_sketch_c64(float2* A, int m, int k, long long sA, int batch, cudaStream_t st) {
    if (batch <= 0 || k <= 0 || m <= 0) return LSW_OK;
    if (k > 64) return LSW_ERR_INVALID_ARG;
    const long long mk = (long long)m * k;
    if (m < 4 * k) {
        DevBuf w;
        LSW_TRY(w.alloc(sizeof(double2) * (size_t)mk * batch, st));
        k_up64<<<grid_small(mk * batch), 256, 0, st>>>(A, sA, w.as<double2>(), mk, batch);
        LSW_LAUNCH_CHECK();
        LSW_TRY(qr_explicit<double>(w.as<double2>(), m, k, mk, batch, nullptr, st));
        k_down32<<<grid_small(mk * batch), 256, 0, st>>>(w.as<double2>(), A, sA, mk, batch);
        LSW_LAUNCH_CHECK();
        return LSW_OK;
    }
    KTimer kt("qr", st, 8.0 * batch * (double)mk * 4, 2.0 * batch * (8.0 * m * k * (k + 1) / 2 * 5 * 2));
    DevBuf G, Ri, flag;
    LSW_TRY(G.alloc(sizeof(double2) * (size_t)batch * k * k, st));
    LSW_TRY(Ri.alloc(sizeof(double2) * (size_t)batch * k * k, st));
    LSW_TRY(flag.alloc(sizeof(int) * (size_t)batch, st));
    static std::atomic<bool> attr{false};
    if (!attr.load()) {
        LSW_CUDA(cudaFuncSetAttribute(k_rmul_dot2, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024));
        attr.store(true);
    }
    const size_t smp = sizeof(float2) * (2 * (size_t)k * k + (size_t)(GT_ROWS + 1) * k);
    const int nchunk = sketch_chunks(m, batch);
    auto pass = [&](const int* active, int* need2) -> lsw_status {
        LSW_TRY(gram64_c64(A, m, k, sA, batch, G.as<double2>(), st, active));
        LSW_TRY(chol_rinv<double>(G.as<double2>(), k, batch, 0.0, Ri.as<double2>(), st, active, need2));
        k_rmul_dot2<<<dim3(nchunk, batch), 256, smp, st>>>(A, m, k, sA, Ri.as<double2>(), active);
        LSW_LAUNCH_CHECK();
        return LSW_OK;
    };
    LSW_TRY(pass(nullptr, flag.as<int>()));
    LSW_TRY(pass(flag.as<int>(), nullptr));
    return LSW_OK;
}

template lsw_status chol_rinv<float>(const double2*, int, int, double, float2*, cudaStream_t, const int*, int*);
template lsw_status chol_rinv<double>(const double2*, int, int, double, double2*, cudaStream_t, const int*, int*);

}  // namespace lsw
