// Dense kernels of the preconditioner build and apply: batched complex GEMM,
// thin Householder QR, FP64 Gram matrices, Jacobi eigen-decomposition of
// small Hermitian matrices, Philox Gaussian probes, blocked Gauss-Jordan
// inversion, norms.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>

#include "lsw_internal.cuh"

namespace lsw {

namespace {

int grid_for(long long n, int bs = 256) {
    long long g = (n + bs - 1) / bs;
    return (int)std::max<long long>(1, std::min<long long>(g, 152LL * 32));
}

template <typename C> __device__ __forceinline__ C ldop(const C* p, bool conj_) {
    C v = *p;
    if (conj_) v.y = -v.y;
    return v;
}

// ------------------------------------------------------------------ GEMM
// BM x BN output tile per CTA, 256 threads, 4 x 4 complex outputs per
// thread, K in steps of 8.  blockIdx.z = batch * ksplit + kpart; with
// ksplit > 1 the partial products go to P (ksplit x batch x m x n) and a
// second kernel reduces them in a fixed order.
constexpr int GBK = 16;

template <typename C, int BM, int BN>
__global__ void __launch_bounds__(256)
k_gemm(int opA, int opB, int m, int n, int k, C alpha, const C* __restrict__ A, int lda, long long sA,
       const C* __restrict__ B, int ldb, long long sB, C beta, C* __restrict__ Cm, int ldc, long long sC,
       int ksplit, int kchunk, C* __restrict__ P) {
    static_assert((BM / 4) * (BN / 4) == 256, "256 threads of 4 x 4 outputs");
    constexpr int TX = BN / 4, TY = BM / 4;
    constexpr int NA = BM * GBK / 256, NB = GBK * BN / 256;
    __shared__ C As[GBK][BM + 1];
    __shared__ C Bs[GBK][BN + 1];
    const int bz = blockIdx.z;
    const int b = bz / ksplit, kp = bz - b * ksplit;
    const int i0 = blockIdx.x * BM, j0 = blockIdx.y * BN;
    const int kbeg = kp * kchunk, kend = min(k, kbeg + kchunk);
    const C* Ab = A + b * sA;
    const C* Bb = B + b * sB;
    const int ty = threadIdx.x % TY, tx = threadIdx.x / TY;   // consecutive lanes: consecutive rows (coalesced C)
    C acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = czero<C>();
    C ra[NA], rb[NB];
    // tile loads into registers (element (i, t) of A's tile, (t, j) of B's)
    auto load = [&](int kk) {
#pragma unroll
        for (int q = 0; q < NA; ++q) {
            const int e = threadIdx.x + 256 * q;
            int i, t;
            if (opA == 0) { i = e % BM; t = e / BM; } else { t = e % GBK; i = e / GBK; }
            const int gi = i0 + i, gk = kk + t;
            C v = czero<C>();
            if (gi < m && gk < kend) v = opA == 0 ? Ab[(long long)gk * lda + gi] : ldop(Ab + (long long)gi * lda + gk, true);
            ra[q] = v;
        }
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int e = threadIdx.x + 256 * q;
            int t, j;
            if (opB == 0) { t = e % GBK; j = e / GBK; } else { j = e % BN; t = e / BN; }
            const int gj = j0 + j, gk = kk + t;
            C v = czero<C>();
            if (gj < n && gk < kend) v = opB == 0 ? Bb[(long long)gj * ldb + gk] : ldop(Bb + (long long)gk * ldb + gj, true);
            rb[q] = v;
        }
    };
    auto store = [&]() {
#pragma unroll
        for (int q = 0; q < NA; ++q) {
            const int e = threadIdx.x + 256 * q;
            int i, t;
            if (opA == 0) { i = e % BM; t = e / BM; } else { t = e % GBK; i = e / GBK; }
            As[t][i] = ra[q];
        }
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int e = threadIdx.x + 256 * q;
            int t, j;
            if (opB == 0) { t = e % GBK; j = e / GBK; } else { j = e % BN; t = e / BN; }
            Bs[t][j] = rb[q];
        }
    };
    if (kbeg < kend) load(kbeg);
    for (int kk = kbeg; kk < kend; kk += GBK) {
        store();
        __syncthreads();
        if (kk + GBK < kend) load(kk + GBK);    // next tile in flight during the products
#pragma unroll
        for (int t = 0; t < GBK; ++t) {
            C a[4], bb[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) { a[q] = As[t][ty + TY * q]; bb[q] = Bs[t][tx + TX * q]; }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) cfma(acc[p][q], a[p], bb[q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int gi = i0 + ty + TY * p, gj = j0 + tx + TX * q;
            if (gi < m && gj < n) {
                if (ksplit == 1) {
                    C* c = Cm + b * sC + (long long)gj * ldc + gi;
                    C r = cmul(alpha, acc[p][q]);
                    if (beta.x != 0 || beta.y != 0) r = cadd(r, cmul(beta, *c));
                    *c = r;
                } else {
                    P[(((long long)kp * gridDim.z / ksplit + b) * n + gj) * m + gi] = acc[p][q];
                }
            }
        }
}

// C = A^H B partial sums for small outputs (m, n <= 64) and long K: CTA
// (kpart, b) takes rows [k0, k1) of A (K x m) and B (K x n) in tiles of 32
// rows through shared memory, stored row-major with odd strides (conflict-
// free transposing stores).  Thread (microtile, row group) keeps a 4 x 4
// block of outputs over every G-th row of a tile; the row groups are summed
// in shared memory at the end.
template <typename C>
__global__ void __launch_bounds__(256)
k_gemm_cn_small(int m, int n, int k, const C* __restrict__ A, int lda, long long sA, const C* __restrict__ B, int ldb,
                long long sB, int kchunk, C* __restrict__ P, int batch) {
    constexpr int TR = 32;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int ms = (m + 3) & ~3, ns = (n + 3) & ~3;
    const int asd = ms + 1, bsd = ns + 1;
    C* As = reinterpret_cast<C*>(sm_raw);         // TR x asd
    C* Bs = As + TR * asd;                         // TR x bsd
    C* Red = Bs + TR * bsd;                        // G x m x n
    const int kp = blockIdx.x, b = blockIdx.y;
    const int k0 = kp * kchunk, k1 = min(k, k0 + kchunk);
    const C* Ab = A + b * sA;
    const C* Bb = B + b * sB;
    const int mtr = ms / 4, mtn = ns / 4, nmt = mtr * mtn;
    const int G = max(1, 256 / nmt);
    const int mt = threadIdx.x % nmt, rg = threadIdx.x / nmt;
    const bool active = rg < G;
    const int i0 = (mt % mtr) * 4, j0 = (mt / mtr) * 4;
    C acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = czero<C>();
    for (int r0 = k0; r0 < k1; r0 += TR) {
        const int nr = min(TR, k1 - r0);
        for (int e = threadIdx.x; e < TR * ms; e += 256) {
            const int cc = e / TR, rr = e - cc * TR;
            As[rr * asd + cc] = (rr < nr && cc < m) ? Ab[(long long)cc * lda + r0 + rr] : czero<C>();
        }
        for (int e = threadIdx.x; e < TR * ns; e += 256) {
            const int cc = e / TR, rr = e - cc * TR;
            Bs[rr * bsd + cc] = (rr < nr && cc < n) ? Bb[(long long)cc * ldb + r0 + rr] : czero<C>();
        }
        __syncthreads();
        if (active) {
            for (int rr = rg; rr < nr; rr += G) {
                C x[4], y[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) x[a] = As[rr * asd + i0 + a];
#pragma unroll
                for (int c = 0; c < 4; ++c) y[c] = Bs[rr * bsd + j0 + c];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 4; ++c) cfmac(acc[a][c], x[a], y[c]);
            }
        }
        __syncthreads();
    }
    const int nout = m * n;
    if (active) {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (i0 + a < m && j0 + c < n) Red[(long long)rg * nout + (j0 + c) * m + i0 + a] = acc[a][c];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nout; e += 256) {
        C sacc = czero<C>();
        for (int g = 0; g < G; ++g) sacc = cadd(sacc, Red[(long long)g * nout + e]);
        P[((long long)kp * batch + b) * nout + e] = sacc;
    }
}

// C = A^H B partial sums for tiny outputs (n <= 4 columns of B): warp w of
// the CTA takes columns i = w, w + 8, ... of A and sums conj(A[r][i]) B[r][j]
// over the CTA's rows with its 32 lanes striding the rows (coalesced), so
// a thread keeps only n accumulators.
template <typename C, int NN>
__global__ void __launch_bounds__(256)
k_gemm_cn_tiny(int m, int k, const C* __restrict__ A, int lda, long long sA, const C* __restrict__ B, int ldb,
               long long sB, int kchunk, C* __restrict__ P, int batch) {
    const int kp = blockIdx.x, b = blockIdx.y;
    const int k0 = kp * kchunk, k1 = min(k, k0 + kchunk);
    const C* Ab = A + b * sA;
    const C* Bb = B + b * sB;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (int i = w; i < m; i += 8) {
        C acc[NN];
#pragma unroll
        for (int j = 0; j < NN; ++j) acc[j] = czero<C>();
        const C* a = Ab + (long long)i * lda;
#pragma unroll 4
        for (int r = k0 + l; r < k1; r += 32) {
            const C av = a[r];
#pragma unroll
            for (int j = 0; j < NN; ++j) cfmac(acc[j], av, Bb[(long long)j * ldb + r]);
        }
#pragma unroll
        for (int j = 0; j < NN; ++j) {
            C v = acc[j];
            for (int o = 16; o > 0; o >>= 1) {
                v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
                v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
            }
            if (l == 0) P[(((long long)kp * batch + b) * NN + j) * m + i] = v;
        }
    }
}

// C = alpha A B + beta C with a small inner dimension (k <= 64) and n <= 64:
// B (k x n) sits in shared memory, thread (row, group of 16 columns) streams
// its row of A.
template <typename C>
__global__ void __launch_bounds__(256)
k_gemm_nn_smallk(int m, int n, int k, C alpha, const C* __restrict__ A, int lda, long long sA, const C* __restrict__ B,
                 int ldb, long long sB, C beta, C* __restrict__ Cm, int ldc, long long sC) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    C* Bs = reinterpret_cast<C*>(sm_raw);       // k x n
    const int b = blockIdx.y;
    const C* Ab = A + b * sA;
    const C* Bb = B + b * sB;
    C* Cb = Cm + b * sC;
    for (int e = threadIdx.x; e < k * n; e += 256) {
        const int j = e / k, t = e - j * k;
        Bs[j * k + t] = Bb[(long long)j * ldb + t];
    }
    __syncthreads();
    const int ngrp = (n + 15) / 16;
    const int rows_per = 256 / ngrp;           // rows handled by this CTA per pass
    const int lr = threadIdx.x % rows_per, g = threadIdx.x / rows_per;
    if (g >= ngrp) return;
    const int i = blockIdx.x * rows_per + lr;
    if (i >= m) return;
    C acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = czero<C>();
    const int j0 = g * 16;
#pragma unroll 4
    for (int t = 0; t < k; ++t) {
        const C a = Ab[(long long)t * lda + i];
#pragma unroll
        for (int q = 0; q < 16; ++q)
            if (j0 + q < n) cfma(acc[q], a, Bs[(j0 + q) * k + t]);
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int j = j0 + q;
        if (j < n) {
            C* c = Cb + (long long)j * ldc + i;
            C r = cmul(alpha, acc[q]);
            if (beta.x != 0 || beta.y != 0) r = cadd(r, cmul(beta, *c));
            *c = r;
        }
    }
}

// y = alpha A b + beta y for a tall A (m x k, k <= 64) and one column b:
// the Krylov-basis updates of the solvers.  A thread owns two consecutive
// rows (one 16-byte load per complex64 row pair) and issues the loads of
// eight columns before their multiply-adds, so a warp keeps 8 x 512 bytes
// in flight.  Requires lda and the A, y pointers even (complex64) for the
// paired loads; the host checks.
template <typename C>
__global__ void __launch_bounds__(256)
k_gemv_tall(int m, int k, C alpha, const C* __restrict__ A, int lda, long long sA, const C* __restrict__ B,
            long long sB, C beta, C* __restrict__ Y, long long sY) {
    __shared__ C bs[64];
    const int b = blockIdx.y;
    const C* Ab = A + b * sA;
    const C* Bb = B + b * sB;
    C* Yb = Y + b * sY;
    for (int t = threadIdx.x; t < k; t += blockDim.x) bs[t] = Bb[t];
    __syncthreads();
    const long long i0 = 2LL * (blockIdx.x * (long long)blockDim.x + threadIdx.x);
    if (i0 >= m) return;
    const bool two = i0 + 1 < m;
    C acc0 = czero<C>(), acc1 = czero<C>();
    for (int t0 = 0; t0 < k; t0 += 8) {
        C a0[8], a1[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int t = t0 + u;
            if (t < k) {
                const C* p = Ab + (long long)t * lda + i0;
                a0[u] = p[0];
                a1[u] = two ? p[1] : czero<C>();
            }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int t = t0 + u;
            if (t < k) {
                cfma(acc0, a0[u], bs[t]);
                cfma(acc1, a1[u], bs[t]);
            }
        }
    }
    C r0 = cmul(alpha, acc0);
    if (beta.x != 0 || beta.y != 0) r0 = cadd(r0, cmul(beta, Yb[i0]));
    Yb[i0] = r0;
    if (two) {
        C r1 = cmul(alpha, acc1);
        if (beta.x != 0 || beta.y != 0) r1 = cadd(r1, cmul(beta, Yb[i0 + 1]));
        Yb[i0 + 1] = r1;
    }
}

template <typename C>
__global__ void k_gemm_reduce(int m, int n, int batch, int ksplit, const C* __restrict__ P, C alpha, C beta,
                              C* __restrict__ Cm, int ldc, long long sC) {
    const long long tot = (long long)batch * m * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(e / ((long long)m * n));
        const long long r = e - (long long)b * m * n;
        const int j = (int)(r / m), i = (int)(r - (long long)j * m);
        C s = czero<C>();
        for (int kp = 0; kp < ksplit; ++kp) s = cadd(s, P[(((long long)kp * batch + b) * n + j) * m + i]);
        C* c = Cm + b * sC + (long long)j * ldc + i;
        C out = cmul(alpha, s);
        if (beta.x != 0 || beta.y != 0) out = cadd(out, cmul(beta, *c));
        *c = out;
    }
}

// ------------------------------------------------------------ FP64 Gram
// G_b = Y_b^H Y_b, k x k (k <= 64), partial sums over row chunks; each
// thread owns up to 16 of the k^2 entries.
template <typename C>
__global__ void __launch_bounds__(256)
k_gram_partial(const C* __restrict__ Y, int m, int k, long long sY, int nchunk, double2* __restrict__ part) {
    constexpr int TR = 32, MAXQ = 16;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    C* sy = reinterpret_cast<C*>(sm_raw);      // k columns of TR rows, stride TR + 1 (odd: lanes on
                                               // different columns hit different banks)
    const int b = blockIdx.y, ch = blockIdx.x;
    const int rows_per = (m + nchunk - 1) / nchunk;
    const int r0 = ch * rows_per, r1 = min(m, r0 + rows_per);
    const C* Yb = Y + b * sY;
    const int npair = k * k;
    double2 acc[MAXQ];
#pragma unroll
    for (int q = 0; q < MAXQ; ++q) acc[q] = make_double2(0, 0);
    for (int rr = r0; rr < r1; rr += TR) {
        const int nr = min(TR, r1 - rr);
        for (int e = threadIdx.x; e < TR * k; e += 256) {
            const int c = e / TR, r = e % TR;
            sy[c * (TR + 1) + r] = r < nr ? Yb[(long long)c * m + rr + r] : czero<C>();
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < MAXQ; ++q) {
            const int pidx = threadIdx.x + q * 256;
            if (pidx < npair) {
                const int i = pidx % k, j = pidx / k;
                const C* yi = sy + i * (TR + 1);
                const C* yj = sy + j * (TR + 1);
                // products and the sum over one tile in the data's precision,
                // tiles accumulated in FP64
                typedef decltype(yi->x) R;
                R sx = 0, syy = 0;
                for (int r = 0; r < nr; ++r) {
                    const R ax = yi[r].x, ay = yi[r].y, bx = yj[r].x, by = yj[r].y;
                    sx = fma(ax, bx, fma(ay, by, sx));
                    syy = fma(ax, by, fma(-ay, bx, syy));
                }
                acc[q] = make_double2(acc[q].x + (double)sx, acc[q].y + (double)syy);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < MAXQ; ++q) {
        const int pidx = threadIdx.x + q * 256;
        if (pidx < npair) part[((long long)b * nchunk + ch) * npair + pidx] = acc[q];
    }
}

__global__ void k_gram_reduce(const double2* __restrict__ part, int nchunk, int npair, int batch, double2* G) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < batch * npair; e += gridDim.x * blockDim.x) {
        const int b = e / npair, p = e - b * npair;
        double2 s = make_double2(0, 0);
        for (int c = 0; c < nchunk; ++c) {
            const double2 v = part[((long long)b * nchunk + c) * npair + p];
            s.x += v.x;
            s.y += v.y;
        }
        G[e] = s;
    }
}

// ------------------------------------------------- Householder QR (thin)
// One CTA per matrix.  Reflectors follow LAPACK's zlarfg convention:
// H = I - tau v v^H with v(0) = 1, H^H [alpha; x] = [beta; 0], beta real.
template <typename C, int NT>
__device__ __forceinline__ C block_sum(C v, C* red) {
    typedef decltype(v.x) R;
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    C s = czero<C>();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : czero<C>();
        for (int o = 16; o > 0; o >>= 1) {
            s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
            s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
        }
        if (threadIdx.x == 0) red[32] = s;
    }
    __syncthreads();
    s = red[32];
    (void)sizeof(R);
    return s;
}

// Warp reduce-scatter: on entry every lane holds 32 values; on exit v[0]
// of lane l is the sum over the warp of value l (31 shuffles per lane).
template <typename C>
__device__ __forceinline__ void warp_reduce_scatter32(C v[32]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const bool upper = (lane & w) != 0;
#pragma unroll
        for (int i = 0; i < w; ++i) {
            const C send = upper ? v[i] : v[i + w];
            const C keep = upper ? v[i + w] : v[i];
            C recv;
            recv.x = __shfl_xor_sync(0xffffffffu, send.x, w);
            recv.y = __shfl_xor_sync(0xffffffffu, send.y, w);
            v[i] = cadd(keep, recv);
        }
    }
}

// CTA sums of up to 32 values per thread: out[c] (shared) = sum over the
// CTA of v[c].  Two barriers.
template <typename C, int NT>
__device__ __forceinline__ void cta_sum32(C v[32], C* red /* [NT/32][32] */, C* out /* [32] */) {
    warp_reduce_scatter32(v);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    red[w * 32 + lane] = v[0];
    __syncthreads();
    if (threadIdx.x < 32) {
        C s = czero<C>();
#pragma unroll
        for (int ww = 0; ww < NT / 32; ++ww) s = cadd(s, red[ww * 32 + threadIdx.x]);
        out[threadIdx.x] = s;
    }
    __syncthreads();
}

// Householder factorisation of A (m x k, ld m, k <= 64) in place, then the
// explicit thin Q.  Rout (k x k, column-major), if given, receives R before
// Q overwrites A.  Works on global or shared memory alike.
//
// Reflectors follow LAPACK's zlarfg convention: H = I - tau v v^H,
// v = [1; s x] with s = 1 / (alpha - beta), H^H [alpha; x] = [beta; 0].
// One pass over the rows below the diagonal gathers ||x||^2 and every
// x^H a_c of the trailing columns together, since
//     v^H a_c = a_c[j] + conj(s) x^H a_c[j+1:],
// so each column costs one CTA reduction; each thread keeps the same rows
// throughout, so the updates need no further barrier.
template <typename R, int NT>
__device__ void hh_qr(typename Cx<R>::T* A, int m, int k, typename Cx<R>::T* Rout) {
    typedef typename Cx<R>::T C;
    __shared__ C red[(NT / 32) * 32];
    __shared__ C sums[32];
    __shared__ C wv[64];          // the reflector's coefficients for the trailing columns
    __shared__ C tau_s[64];
    __shared__ C hdr[3];          // tau, s, beta of the current column
    const int kk = min(k, m);
    // ---- factorisation
    for (int j = 0; j < kk; ++j) {
        C* aj = A + (long long)j * m;
        // trailing columns in groups of 31 (slot 31 of the first group: ||x||^2)
        for (int g0 = j + 1, first = 1; first || g0 < k; g0 += 31, first = 0) {
            const int nc = min(31, k - g0);
            C acc[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) acc[q] = czero<C>();
            for (int i = threadIdx.x; i < m; i += NT) {
                if (i <= j) continue;
                const C x = aj[i];
                if (first) acc[31].x += x.x * x.x + x.y * x.y;
#pragma unroll
                for (int q = 0; q < 31; ++q)
                    if (q < nc) cfmac(acc[q], x, A[(long long)(g0 + q) * m + i]);
            }
            cta_sum32<C, NT>(acc, red, sums);
            if (first && threadIdx.x == 0) {
                const C alpha = aj[j];
                const R xnorm2 = sums[31].x;
                C tau = czero<C>(), scale = czero<C>();
                R beta = alpha.x;
                if (!(xnorm2 == 0 && alpha.y == 0)) {
                    const R nrm = sqrt(alpha.x * alpha.x + alpha.y * alpha.y + xnorm2);
                    beta = alpha.x >= 0 ? -nrm : nrm;
                    tau = mk((beta - alpha.x) / beta, -alpha.y / beta);
                    const C d = mk(alpha.x - beta, alpha.y);
                    const R den = d.x * d.x + d.y * d.y;
                    scale = mk(d.x / den, -d.y / den);
                }
                hdr[0] = tau;
                hdr[1] = scale;
                hdr[2] = mk(beta, (R)0);
                tau_s[j] = tau;
            }
            if (first) __syncthreads();
            // v^H a_c = a_c[j] + conj(s) (x^H a_c);  wv_c = conj(tau) v^H a_c
            if (threadIdx.x < nc) {
                const C ajc = A[(long long)(g0 + threadIdx.x) * m + j];
                wv[g0 + threadIdx.x - j - 1] = cmulc(hdr[0], cadd(ajc, cmulc(hdr[1], sums[threadIdx.x])));
            }
            __syncthreads();   // wv complete, row j read by all before any update
            if (nc <= 0) break;
        }
        const C tau = hdr[0], scale = hdr[1];
        const R beta = hdr[2].x;
        const bool skip = tau.x == 0 && tau.y == 0;
        if (!skip) {
            for (int i = threadIdx.x; i < m; i += NT) {
                if (i < j) continue;
                if (i == j) {
                    for (int c = j + 1; c < k; ++c) {
                        C* a = A + (long long)c * m + j;
                        *a = csub(*a, wv[c - j - 1]);
                    }
                    continue;
                }
                const C v = cmul(aj[i], scale);
                aj[i] = v;
                for (int c = j + 1; c < k; ++c) {
                    C* a = A + (long long)c * m + i;
                    *a = csub(*a, cmul(v, wv[c - j - 1]));
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) aj[j] = mk(beta, (R)0);
    }
    __syncthreads();
    if (Rout) {
        for (int e = threadIdx.x; e < k * k; e += NT) {
            const int jj = e / k, i = e - jj * k;
            Rout[e] = (i <= jj && i < kk) ? A[(long long)jj * m + i] : czero<C>();
        }
        __syncthreads();
    }
    // ---- explicit Q = H_0 H_1 ... H_{k-1} [I; 0]
    for (int j = k - 1; j >= 0; --j) {
        C* aj = A + (long long)j * m;
        if (j >= kk) {          // more columns than rows: column j of Q is zero
            for (int i = threadIdx.x; i < m; i += NT) aj[i] = czero<C>();
            __syncthreads();
            continue;
        }
        const C tau = tau_s[j];
        // w_c = tau v^H q_c = tau (q_c[j] + sum_{i>j} conj(v_i) q_c[i])
        for (int g0 = j + 1; g0 < k; g0 += 32) {
            const int nc = min(32, k - g0);
            C acc[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) acc[q] = czero<C>();
            for (int i = threadIdx.x; i < m; i += NT) {
                if (i <= j) continue;
                const C v = aj[i];
#pragma unroll
                for (int q = 0; q < 32; ++q)
                    if (q < nc) cfmac(acc[q], v, A[(long long)(g0 + q) * m + i]);
            }
            cta_sum32<C, NT>(acc, red, sums);
            if (threadIdx.x < nc)
                wv[g0 + threadIdx.x - j - 1] = cmul(tau, cadd(A[(long long)(g0 + threadIdx.x) * m + j], sums[threadIdx.x]));
            __syncthreads();
        }
        for (int i = threadIdx.x; i < m; i += NT) {
            if (i < j) { aj[i] = czero<C>(); continue; }
            const C v = i == j ? mk((R)1, (R)0) : aj[i];
            for (int c = j + 1; c < k; ++c) {
                C* a = A + (long long)c * m + i;
                *a = csub(*a, cmul(v, wv[c - j - 1]));
            }
            aj[i] = i == j ? mk((R)1 - tau.x, -tau.y) : mk(-(tau.x * v.x - tau.y * v.y), -(tau.x * v.y + tau.y * v.x));
        }
        __syncthreads();
    }
}

// The same factorisation for k <= 32 columns and m <= 2 NT rows (every
// thread owns rows t and t + NT), with each column's update fused into the
// pass that gathers the next column's reductions:
//   factorisation: every thread forms the reflector of column j from the
//     sums (alpha, ||x||^2, x^H a_c); threads t < k - j - 1 put
//     w_c = conj(tau) v^H a_c in shared memory and R's row j in Rout (row j
//     of A is not written during step j); one pass then scales v, updates
//     the trailing columns of each row and accumulates ||x'||^2 and x'^H a'_c
//     of the next column;
//   explicit Q = H_0 ... H_{k-1} [I; 0], from j = k-1 down: rows < j of the
//     columns > j are still zero, so w_c = tau v_j^H q_c is tau times the
//     sums of the previous pass; one pass forms column j, updates columns
//     > j and accumulates v_{j-1}^H q_c for the next step.
// One pass per column in each half (hh_qr makes two), three and two
// barriers per column (hh_qr four and three); the arithmetic and its order
// are the same.  Rout (k x k, column-major) is required.
template <typename R, int NT>
__device__ void hh_qr32(typename Cx<R>::T* A, int m, int k, typename Cx<R>::T* Rout) {
    typedef typename Cx<R>::T C;
    __shared__ C red[(NT / 32) * 32];
    __shared__ C sums[32];
    __shared__ C wv[32];
    __shared__ C tau_s[32];
    const int kk = min(k, m);
    for (int e = threadIdx.x; e < k * k; e += NT) Rout[e] = czero<C>();
    C acc[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) acc[q] = czero<C>();
    // column 0: ||x||^2 in slot 31, x^H a_c in slot c - 1
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const int i = threadIdx.x + s * NT;
        if (i >= m || i == 0) continue;
        const C x = A[i];
        acc[31].x += x.x * x.x + x.y * x.y;
#pragma unroll
        for (int q = 0; q < 31; ++q)
            if (q < k - 1) cfmac(acc[q], x, A[(long long)(1 + q) * m + i]);
    }
    cta_sum32<C, NT>(acc, red, sums);
    // ---- factorisation
    for (int j = 0; j < kk; ++j) {
        const int nc = k - j - 1;
        const C alpha = A[(long long)j * m + j];
        const R xnorm2 = sums[31].x;
        C tau = czero<C>(), scale = czero<C>();
        R beta = alpha.x;
        if (!(xnorm2 == 0 && alpha.y == 0)) {
            const R nrm = sqrt(alpha.x * alpha.x + alpha.y * alpha.y + xnorm2);
            beta = alpha.x >= 0 ? -nrm : nrm;
            tau = mk((beta - alpha.x) / beta, -alpha.y / beta);
            const C d = mk(alpha.x - beta, alpha.y);
            const R den = d.x * d.x + d.y * d.y;
            scale = mk(d.x / den, -d.y / den);
        }
        if (threadIdx.x < nc) {
            // w_c = conj(tau) (a_c[j] + conj(s) x^H a_c), c = j + 1 + t
            const int t = threadIdx.x;
            const C ajc = A[(long long)(j + 1 + t) * m + j];
            const C w = cmulc(tau, cadd(ajc, cmulc(scale, sums[t])));
            wv[t] = w;
            Rout[(j + 1 + t) * k + j] = csub(ajc, w);
        }
        if (threadIdx.x == 0) {
            Rout[j * k + j] = mk(beta, (R)0);
            tau_s[j] = tau;
        }
        __syncthreads();   // wv complete
#pragma unroll
        for (int q = 0; q < 32; ++q) acc[q] = czero<C>();
        C v[2], x[2];
        bool act[2], nxt[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int i = threadIdx.x + s * NT;
            act[s] = i < m && i > j;
            nxt[s] = act[s] && i > j + 1;
            v[s] = x[s] = czero<C>();
            if (act[s]) {
                v[s] = cmul(A[(long long)j * m + i], scale);
                A[(long long)j * m + i] = v[s];
            }
        }
        if (nc > 0) {
            const C w0 = wv[0];
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                if (!act[s]) continue;
                C* a = A + (long long)(j + 1) * m + threadIdx.x + s * NT;
                x[s] = csub(*a, cmul(v[s], w0));
                *a = x[s];
                if (nxt[s]) acc[31].x += x[s].x * x[s].x + x[s].y * x[s].y;
            }
            // columns in groups of four without a branch inside a group (four
            // independent chains): a slot past the last column rewrites
            // column k - 1 unchanged (w = 0) after its real update, and its
            // sum is not kept
#pragma unroll
            for (int q0 = 0; q0 < 30; q0 += 4) {
                if (q0 < nc - 1) {
#pragma unroll
                    for (int d = 0; d < 4; ++d) {
                        const int q = q0 + d;
                        if (q >= 30) break;
                        const bool ok = q < nc - 1;
                        const int col = ok ? j + 2 + q : k - 1;
                        const C w = ok ? wv[q + 1] : czero<C>();
#pragma unroll
                        for (int s = 0; s < 2; ++s) {
                            if (!act[s]) continue;
                            C* a = A + (long long)col * m + threadIdx.x + s * NT;
                            const C y = csub(*a, cmul(v[s], w));
                            *a = y;
                            if (nxt[s] && ok) cfmac(acc[q], x[s], y);
                        }
                    }
                }
            }
        }
        if (j + 1 < kk) cta_sum32<C, NT>(acc, red, sums);   // its first barrier also retires wv
        else __syncthreads();
    }
    // ---- explicit Q; columns kk.. are zero (more columns than rows)
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const int i = threadIdx.x + s * NT;
        if (i < m)
            for (int c = kk; c < k; ++c) A[(long long)c * m + i] = czero<C>();
    }
    for (int j = kk - 1; j >= 0; --j) {
        const C tau = tau_s[j];
        const int nc = k - j - 1;
#pragma unroll
        for (int q = 0; q < 32; ++q) acc[q] = czero<C>();
        C v[2], vn[2];
        bool act[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int i = threadIdx.x + s * NT;
            act[s] = i < m && i >= j;
            v[s] = vn[s] = czero<C>();
            if (i < m && i < j) A[(long long)j * m + i] = czero<C>();
            if (!act[s]) continue;
            C* aj = A + (long long)j * m + i;
            v[s] = i == j ? mk((R)1, (R)0) : *aj;
            const C qj = i == j ? mk((R)1 - tau.x, -tau.y)
                                : mk(-(tau.x * v[s].x - tau.y * v[s].y), -(tau.x * v[s].y + tau.y * v[s].x));
            *aj = qj;
            if (j > 0) {
                vn[s] = A[(long long)(j - 1) * m + i];
                cfmac(acc[0], vn[s], qj);
            }
        }
        if (j < kk - 1) {   // the columns > j hold Q's partial product
            // groups of four as in the factorisation (a slot past the last
            // column rewrites column k - 1 unchanged)
#pragma unroll
            for (int q0 = 0; q0 < 31; q0 += 4) {
                if (q0 < nc) {
#pragma unroll
                    for (int d = 0; d < 4; ++d) {
                        const int q = q0 + d;
                        if (q >= 31) break;
                        const bool ok = q < nc;
                        const int col = ok ? j + 1 + q : k - 1;
                        const C w = ok ? cmul(tau, sums[q]) : czero<C>();
#pragma unroll
                        for (int s = 0; s < 2; ++s) {
                            if (!act[s]) continue;
                            C* a = A + (long long)col * m + threadIdx.x + s * NT;
                            const C y = csub(*a, cmul(v[s], w));
                            *a = y;
                            if (j > 0 && ok) cfmac(acc[q + 1], vn[s], y);
                        }
                    }
                }
            }
        }
        if (j > 0) cta_sum32<C, NT>(acc, red, sums);
    }
    __syncthreads();
}

// Chunk step of TSQR: rows [r0, r1) of block b (chunk ch of nch, sizes as
// even as possible) are factored in shared memory; Q_chunk replaces them and
// R_chunk goes to rows ch*k.. of the stacked matrix S_b ((nch*k) x k).
template <typename R, int NT>
__global__ void __launch_bounds__(NT)
k_tsqr_chunk(typename Cx<R>::T* __restrict__ Aall, int m, int k, long long sA, int nch,
             typename Cx<R>::T* __restrict__ Sall) {
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int b = blockIdx.y, ch = blockIdx.x;
    const long long r0 = (long long)m * ch / nch, r1 = (long long)m * (ch + 1) / nch;
    const int cc = (int)(r1 - r0);
    C* Rs = reinterpret_cast<C*>(sm_raw);            // k x k
    C* As = Rs + k * k;                               // cc x k
    C* A = Aall + b * sA;
    for (int e = threadIdx.x; e < cc * k; e += NT) {
        const int j = e / cc, i = e - j * cc;
        As[e] = A[(long long)j * m + r0 + i];
    }
    __syncthreads();
    // (FP64 at 512 threads keeps hh_qr: 32 double2 sums already fill the
    // 128 registers a thread has there)
    if constexpr (sizeof(R) == 4 || NT <= 128) {
        if (k <= 32 && cc <= 2 * NT) {
            hh_qr32<R, NT>(As, cc, k, Rs);
        } else {
            hh_qr<R, NT>(As, cc, k, Rs);
        }
    } else {
        hh_qr<R, NT>(As, cc, k, Rs);
    }
    const int ms = nch * k;
    C* S = Sall + (long long)b * ms * k;
    for (int e = threadIdx.x; e < k * k; e += NT) {
        const int j = e / k, i = e - j * k;
        S[(long long)j * ms + ch * k + i] = Rs[e];
    }
    for (int e = threadIdx.x; e < cc * k; e += NT) {
        const int j = e / cc, i = e - j * cc;
        A[(long long)j * m + r0 + i] = As[e];
    }
}

// Final TSQR step: Q_rows(chunk) = Q_chunk * Qtop[ch*k : ch*k + k, :].
template <typename R, int NT>
__global__ void __launch_bounds__(NT)
k_tsqr_apply(typename Cx<R>::T* __restrict__ Aall, int m, int k, long long sA, int nch,
             const typename Cx<R>::T* __restrict__ Sall) {
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int b = blockIdx.y, ch = blockIdx.x;
    const long long r0 = (long long)m * ch / nch, r1 = (long long)m * (ch + 1) / nch;
    const int cc = (int)(r1 - r0);
    C* Ts = reinterpret_cast<C*>(sm_raw);            // k x k
    C* As = Ts + k * k;                               // cc x k
    C* A = Aall + b * sA;
    const int ms = nch * k;
    const C* S = Sall + (long long)b * ms * k;
    for (int e = threadIdx.x; e < k * k; e += NT) {
        const int j = e / k, i = e - j * k;
        Ts[e] = S[(long long)j * ms + ch * k + i];
    }
    for (int e = threadIdx.x; e < cc * k; e += NT) {
        const int j = e / cc, i = e - j * cc;
        As[e] = A[(long long)j * m + r0 + i];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < cc * k; e += NT) {
        const int j = e / cc, i = e - j * cc;
        C acc = czero<C>();
        for (int t = 0; t < k; ++t) cfma(acc, As[t * cc + i], Ts[j * k + t]);
        A[(long long)j * m + r0 + i] = acc;
    }
}

// --------------------------------------------- Jacobi eigen (Hermitian)
// A pair (p, q) is rotated only while |a_pq| > t sqrt(|a_pp a_qq|), t a few
// units of rounding of the working precision; a sweep that rotates nothing
// ends the iteration (the classical threshold rule, which terminates even
// when rounding keeps the off-diagonal norm above a fixed fraction).
template <typename R> __device__ __forceinline__ R jacobi_skip() { return sizeof(R) == 8 ? (R)1e-14 : (R)1e-6; }

// Parallel cyclic Jacobi in precision R: each round rotates k/2 disjoint
// index pairs chosen by the circle method, so every pair is met once per
// sweep.  Input: FP64 Hermitian G (k x k), scaled by its trace; output: the
// eigenvectors as columns of V, by decreasing eigenvalue.
// sort key of an eigenvalue: a NaN sorts last, so that the ranks of any k
// values (ties broken by index) are a permutation of 0 .. k-1
template <typename R>
__device__ __forceinline__ R jacobi_key(R d) { return isnan(d) ? -INFINITY : d; }

#define JACOBI_MARK_ROUND (rf[r & 1] = 1)
template <typename R>
__global__ void __launch_bounds__(1024)
k_heev_jacobi(const double2* __restrict__ Gall, typename Cx<R>::T* __restrict__ Vall, int k, int polish) {
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int m = (k + 1) & ~1;                 // even number of players
    C* A = reinterpret_cast<C*>(sm_raw);        // k x k, column-major
    C* A2 = A + k * k;                          // the next round's A
    C* V = A2 + k * k;
    R* rot = reinterpret_cast<R*>(V + k * k);   // per pair: cs, sn, cos(phi), sin(phi)
    int2* pr = reinterpret_cast<int2*>(rot + 4 * (m / 2));
    __shared__ C red[33];
    __shared__ double trs;
    __shared__ int order[64];
    __shared__ int nrot;
    // the 2 x 2 blocks (pair i, pair j), i <= j, of a round's update
    __shared__ short2 blk[32 * 33 / 2];
    const int nbt = (m / 2) * (m / 2 + 1) / 2;
    for (int t = threadIdx.x; t < nbt; t += blockDim.x) {
        int j = 0;
        while ((j + 1) * (j + 2) / 2 <= t) ++j;
        blk[t] = make_short2((short)(t - j * (j + 1) / 2), (short)j);
    }
    const double2* G = Gall + (long long)blockIdx.x * k * k;
    // e / k for e < k * k <= 4096 by a multiply and a shift (exact for k < 256)
    const unsigned kinv = (1u << 20) / (unsigned)k + 1u;
    const unsigned khinv = (1u << 20) / (unsigned)((k + 1) >> 1) + 1u;
    if (threadIdx.x < 32) {
        double t = 0;
        for (int i = threadIdx.x; i < k; i += 32) t += fabs(G[i * k + i].x);
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) trs = t > 0 ? 1.0 / t : 0.0;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
        A[e] = mk((R)(G[e].x * trs), (R)(G[e].y * trs));
        V[e] = mk((R)((e % k) == (e / k) ? 1 : 0), (R)0);
    }
    __syncthreads();
    // squared off-diagonal norm relative to the total that the precision
    // can reach (FP32 rounding stalls near 1e-13): stop there.  A polishing
    // run (a nearly diagonal input whose small eigenvalues must be resolved
    // relative to themselves) stops only on a sweep without rotations and
    // uses a tighter pair threshold.
    // polish 2 (coarse): a first pass that a polish run will finish
    const R tol = polish == 1 ? (R)0 : polish == 2 ? (R)1e-6 : (sizeof(R) == 8 ? (R)1e-26 : (R)1e-11);
    const R skip = polish == 1 ? (sizeof(R) == 8 ? (R)1e-15 : (R)2e-7) : jacobi_skip<R>();
    // the trace-scaled input is known to ~1e-16 absolute (an FP64-accurate
    // matrix): entries below that are noise and never trigger a rotation, so
    // a polish of a matrix with (near-)zero eigenvalues still ends
    const R floor_abs = polish == 1 ? (R)1e-15 : (R)0;
    __shared__ int rf[2];               // per round (alternating): some pair rotates
    for (int sweep = 0; sweep < (polish == 1 ? 20 : 40); ++sweep) {
        // both flags clear before the sweep's first round (the block sum
        // below synchronises; the previous round's reads ended at its last barrier)
        if (threadIdx.x < 2) rf[threadIdx.x] = 0;
        C part = czero<C>();
        int need = 0;                   // some pair is above the rotation threshold
        for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
            const C a = A[e];
            const R v = a.x * a.x + a.y * a.y;
            part.y += v;
            const int b = (int)(((unsigned)e * kinv) >> 20), aa = e - b * k;
            if (aa != b) {
                part.x += v;
                if (aa < b) {
                    const R app = A[aa * k + aa].x, aqq = A[b * k + b].x, ac = sqrt(v);
                    if (ac > skip * sqrt(fabs(app * aqq)) && ac > (R)1e-30 * (fabs(app) + fabs(aqq)) &&
                        ac > floor_abs && ac > 0)
                        need = 1;
                }
            }
        }
        const C on = block_sum<C, 1024>(part, red);
        if (!(on.x > tol * on.y) || on.y == 0) break;
        if (!__syncthreads_or(need)) break;     // no pair would rotate: converged
        if (threadIdx.x == 0) nrot = 0;
        for (int r = 0; r < m - 1; ++r) {
            for (int i = threadIdx.x; i < m / 2; i += blockDim.x) {
                int p, q;
                if (i == 0) { p = m - 1; q = r; }
                else {
                    // (r + i) mod (m - 1) and (r - i) mod (m - 1): both below 2 (m - 1)
                    p = r + i;
                    if (p >= m - 1) p -= m - 1;
                    q = r - i + (m - 1);
                    if (q >= m - 1) q -= m - 1;
                }
                if (p > q) { const int t = p; p = q; q = t; }
                R cs = 1, sn = 0, cp = 1, spp = 0;
                if (q < k) {
                    const R app = A[p * k + p].x, aqq = A[q * k + q].x;
                    const C c = A[q * k + p];   // A[p][q]
                    const R ac2 = c.x * c.x + c.y * c.y, ac = sqrt(ac2);
                    // rotate only while the pair is not yet negligible
                    // against its diagonal (relative threshold above rounding)
                    if (ac > skip * sqrt(fabs(app * aqq)) && ac > (R)1e-30 * (fabs(app) + fabs(aqq)) &&
                        ac > floor_abs && ac > 0) {
                        nrot = 1;
                        JACOBI_MARK_ROUND;
                        // t = tan(theta) = sign(d) 2|a_pq| / (|d| + sqrt(d^2 + 4|a_pq|^2)),
                        // d = a_qq - a_pp: the smaller root of t^2 + (d / |a_pq|) t - 1 = 0
                        const R d = aqq - app;
                        const R t = (d >= 0 ? (R)2 : (R)-2) * ac / (fabs(d) + sqrt(d * d + 4 * ac2));
                        const R rac = (R)1 / ac;
                        cs = (R)1 / sqrt((R)1 + t * t);
                        sn = t * cs;
                        cp = c.x * rac;
                        spp = c.y * rac;
                    }
                }
                rot[4 * i] = cs; rot[4 * i + 1] = sn; rot[4 * i + 2] = cp; rot[4 * i + 3] = spp;
                pr[i] = make_int2(p, q);
            }
            __syncthreads();
            // a round without a rotation leaves A and V as they are
            const bool any = rf[r & 1] != 0;
            if (threadIdx.x == 0) rf[(r + 1) & 1] = 0;
            // U on pair (p, q): col p = cs e_p - sn e^{-i phi} e_q, col q = sn e_p
            // + cs e^{-i phi} e_q, i.e. the 2 x 2 block J = [cs, sn; -sn em, cs em]
            // (em = e^{-i phi}).  A <- U^H A U by 2 x 2 blocks, one item per
            // pair of pairs i <= j from the old A into the other buffer:
            //   A'[{p,q}, {p',q'}] = J_i^H A[{p,q}, {p',q'}] J_j,
            // the block (j, i) its conjugate transpose; the index beyond k (odd
            // k) has no row or column.  V <- V U in place, one row of a pair of
            // columns per item.
            const int kh = (k + 1) >> 1;                    // row pairs of V
            const int nvt = (m / 2) * kh;
            for (int t = threadIdx.x; any && t < nbt + nvt; t += blockDim.x) {
                if (t < nbt) {
                    const short2 ij = blk[t];
                    const int i = ij.x, j = ij.y;
                    const int p = pr[i].x, q = pr[i].y, p2 = pr[j].x, q2 = pr[j].y;
                    const bool hq = q < k, hq2 = q2 < k;
                    const R c1 = rot[4 * i], s1 = rot[4 * i + 1], c2 = rot[4 * j], s2 = rot[4 * j + 1];
                    const C ep1 = mk(rot[4 * i + 2], rot[4 * i + 3]);    // conj(em) of pair i
                    const C em2 = mk(rot[4 * j + 2], -rot[4 * j + 3]);   // em of pair j
                    const C b00 = A[p2 * k + p];
                    const C b01 = hq2 ? A[q2 * k + p] : czero<C>();
                    const C b10 = hq ? A[p2 * k + q] : czero<C>();
                    const C b11 = (hq && hq2) ? A[q2 * k + q] : czero<C>();
                    // T = J_i^H B:  row p: cs b0x - sn ep b1x,  row q: sn b0x + cs ep b1x
                    const C e10 = cmul(ep1, b10), e11 = cmul(ep1, b11);
                    const C t00 = mk(c1 * b00.x - s1 * e10.x, c1 * b00.y - s1 * e10.y);
                    const C t01 = mk(c1 * b01.x - s1 * e11.x, c1 * b01.y - s1 * e11.y);
                    const C t10 = mk(s1 * b00.x + c1 * e10.x, s1 * b00.y + c1 * e10.y);
                    const C t11 = mk(s1 * b01.x + c1 * e11.x, s1 * b01.y + c1 * e11.y);
                    // B' = T J_j:  col p': cs' Tx0 - sn' em' Tx1,  col q': sn' Tx0 + cs' em' Tx1
                    const C f01 = cmul(t01, em2), f11 = cmul(t11, em2);
                    C n00 = mk(c2 * t00.x - s2 * f01.x, c2 * t00.y - s2 * f01.y);
                    C n01 = mk(s2 * t00.x + c2 * f01.x, s2 * t00.y + c2 * f01.y);
                    C n10 = mk(c2 * t10.x - s2 * f11.x, c2 * t10.y - s2 * f11.y);
                    C n11 = mk(s2 * t10.x + c2 * f11.x, s2 * t10.y + c2 * f11.y);
                    if (i == j) {
                        // the diagonal block: the entry the rotation annihilates is zero
                        if (s1 != (R)0) { n01 = czero<C>(); n10 = czero<C>(); }
                        A2[p * k + p] = n00;
                        if (hq) { A2[q * k + p] = n01; A2[p * k + q] = n10; A2[q * k + q] = n11; }
                    } else {
                        A2[p2 * k + p] = n00;
                        A2[p * k + p2] = cconj(n00);
                        if (hq2) { A2[q2 * k + p] = n01; A2[p * k + q2] = cconj(n01); }
                        if (hq) { A2[p2 * k + q] = n10; A2[q * k + p2] = cconj(n10); }
                        if (hq && hq2) { A2[q2 * k + q] = n11; A2[q * k + q2] = cconj(n11); }
                    }
                } else {
                    const int e = t - nbt;
                    const int i = (int)(((unsigned)e * khinv) >> 20), r0 = 2 * (e - i * kh);
                    const int p = pr[i].x, q = pr[i].y;
                    if (q >= k) continue;
                    const R cs = rot[4 * i], sn = rot[4 * i + 1];
                    const C em = mk(rot[4 * i + 2], -rot[4 * i + 3]);   // e^{-i phi}
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int row = r0 + u;
                        if (row < k) {
                            const C vp = V[p * k + row], eq = cmul(em, V[q * k + row]);
                            V[p * k + row] = mk(cs * vp.x - sn * eq.x, cs * vp.y - sn * eq.y);
                            V[q * k + row] = mk(sn * vp.x + cs * eq.x, sn * vp.y + cs * eq.y);
                        }
                    }
                }
            }
            __syncthreads();
            if (any) { C* t = A; A = A2; A2 = t; }
        }
        if (nrot == 0) break;          // a sweep without a rotation: converged
        __syncthreads();
    }
    // descending order of the eigenvalues (ties by index): index i goes to
    // the position given by its rank
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        const R di = jacobi_key(A[i * k + i].x);
        int pos = 0;
        for (int j = 0; j < k; ++j) {
            const R dj = jacobi_key(A[j * k + j].x);
            pos += (dj > di || (dj == di && j < i)) ? 1 : 0;
        }
        order[pos] = i;
    }
    __syncthreads();
    C* Vo = Vall + (long long)blockIdx.x * k * k;
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
        const int col = e / k, row = e - col * k;
        Vo[e] = V[order[col] * k + row];
    }
}

// The same Jacobi iteration with one warp per matrix (k <= 64) and several
// matrices per CTA: lanes share the work of a round, __syncwarp orders it.
#undef JACOBI_MARK_ROUND
#define JACOBI_COUNT_ROTATION ++nrw
#define JACOBI_MARK_ROUND (rr = 1)
template <typename R>
__global__ void __launch_bounds__(256)
k_heev_jacobi_warp(const double2* __restrict__ Gall, typename Cx<R>::T* __restrict__ Vall, int k, int batch,
                   int polish) {
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int m = (k + 1) & ~1;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mat = blockIdx.x * (blockDim.x >> 5) + w;
    const size_t per = sizeof(C) * 2 * k * k + sizeof(R) * 4 * (m / 2) + sizeof(int2) * (m / 2) + sizeof(int) * 64;
    const size_t perA = (per + 15) & ~size_t(15);
    unsigned char* base = sm_raw + perA * w;
    C* A = reinterpret_cast<C*>(base);
    C* V = A + k * k;
    R* rot = reinterpret_cast<R*>(V + k * k);
    int2* pr = reinterpret_cast<int2*>(rot + 4 * (m / 2));
    int* order = reinterpret_cast<int*>(pr + m / 2);
    if (mat >= batch) return;           // whole warp leaves together
    const double2* G = Gall + (long long)mat * k * k;
    double tr = 0;
    for (int i = lane; i < k; i += 32) tr += fabs(G[i * k + i].x);
    for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
    const double trs = tr > 0 ? 1.0 / tr : 0.0;
    for (int e = lane; e < k * k; e += 32) {
        A[e] = mk((R)(G[e].x * trs), (R)(G[e].y * trs));
        V[e] = mk((R)((e % k) == (e / k) ? 1 : 0), (R)0);
    }
    __syncwarp();
    // the same stopping rules as the CTA version
    // polish 2 (coarse): a first pass that a polish run will finish
    const R tol = polish == 1 ? (R)0 : polish == 2 ? (R)1e-6 : (sizeof(R) == 8 ? (R)1e-26 : (R)1e-11);
    const R skip = polish == 1 ? (sizeof(R) == 8 ? (R)1e-15 : (R)2e-7) : jacobi_skip<R>();
    // the trace-scaled input is known to ~1e-16 absolute (an FP64-accurate
    // matrix): entries below that are noise and never trigger a rotation, so
    // a polish of a matrix with (near-)zero eigenvalues still ends
    const R floor_abs = polish == 1 ? (R)1e-15 : (R)0;
    for (int sweep = 0; sweep < (polish == 1 ? 20 : 40); ++sweep) {
        R off = 0, tot = 0;
        int need = 0;                   // some pair is above the rotation threshold
        for (int e = lane; e < k * k; e += 32) {
            const C a = A[e];
            const R v = a.x * a.x + a.y * a.y;
            tot += v;
            const int b = e / k, aa = e - b * k;
            if (aa != b) {
                off += v;
                if (aa < b) {
                    const R app = A[aa * k + aa].x, aqq = A[b * k + b].x, ac = sqrt(v);
                    if (ac > skip * sqrt(fabs(app * aqq)) && ac > (R)1e-30 * (fabs(app) + fabs(aqq)) &&
                        ac > floor_abs && ac > 0)
                        need = 1;
                }
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            tot += __shfl_xor_sync(0xffffffffu, tot, o);
        }
        if (!(off > tol * tot) || tot == 0) break;
        if (!__any_sync(0xffffffffu, need)) break;   // no pair would rotate: converged
        int nrw = 0;
        for (int r = 0; r < m - 1; ++r) {
            int rr = 0;
            for (int i = lane; i < m / 2; i += 32) {
                int p, q;
                if (i == 0) { p = m - 1; q = r; }
                else { p = (r + i) % (m - 1); q = (r - i + (m - 1)) % (m - 1); }
                if (p > q) { const int t = p; p = q; q = t; }
                R cs = 1, sn = 0, cp = 1, spp = 0;
                if (q < k) {
                    const R app = A[p * k + p].x, aqq = A[q * k + q].x;
                    const C c = A[q * k + p];
                    const R ac2 = c.x * c.x + c.y * c.y, ac = sqrt(ac2);
                    // rotate only while the pair is not yet negligible
                    // against its diagonal (relative threshold above rounding)
                    if (ac > skip * sqrt(fabs(app * aqq)) && ac > (R)1e-30 * (fabs(app) + fabs(aqq)) &&
                        ac > floor_abs && ac > 0) {
                        JACOBI_COUNT_ROTATION;
                        JACOBI_MARK_ROUND;
                        // the same rotation as the CTA version
                        const R d = aqq - app;
                        const R t = (d >= 0 ? (R)2 : (R)-2) * ac / (fabs(d) + sqrt(d * d + 4 * ac2));
                        const R rac = (R)1 / ac;
                        cs = (R)1 / sqrt((R)1 + t * t);
                        sn = t * cs;
                        cp = c.x * rac;
                        spp = c.y * rac;
                    }
                }
                rot[4 * i] = cs; rot[4 * i + 1] = sn; rot[4 * i + 2] = cp; rot[4 * i + 3] = spp;
                pr[i] = make_int2(p, q);
            }
            // a round without a rotation leaves A and V as they are
            if (!__any_sync(0xffffffffu, rr)) continue;
            __syncwarp();
            for (int e = lane; e < (m / 2) * k; e += 32) {
                const int i = e / k, row = e - i * k;
                const int p = pr[i].x, q = pr[i].y;
                if (q >= k) continue;
                const R cs = rot[4 * i], sn = rot[4 * i + 1];
                const C em = mk(rot[4 * i + 2], -rot[4 * i + 3]);
                for (int ww = 0; ww < 2; ++ww) {
                    C* M = ww ? V : A;
                    const C ap = M[p * k + row], aq = M[q * k + row];
                    const C eq = cmul(em, aq);
                    M[p * k + row] = mk(cs * ap.x - sn * eq.x, cs * ap.y - sn * eq.y);
                    M[q * k + row] = mk(sn * ap.x + cs * eq.x, sn * ap.y + cs * eq.y);
                }
            }
            __syncwarp();
            for (int e = lane; e < (m / 2) * k; e += 32) {
                const int i = e / k, col = e - i * k;
                const int p = pr[i].x, q = pr[i].y;
                if (q >= k) continue;
                const R cs = rot[4 * i], sn = rot[4 * i + 1];
                const C ep = mk(rot[4 * i + 2], rot[4 * i + 3]);
                const C ap = A[col * k + p], aq = A[col * k + q];
                const C eq = cmul(ep, aq);
                A[col * k + p] = mk(cs * ap.x - sn * eq.x, cs * ap.y - sn * eq.y);
                A[col * k + q] = mk(sn * ap.x + cs * eq.x, sn * ap.y + cs * eq.y);
            }
            __syncwarp();
            // the entries a rotation annihilates are zero by construction
            for (int i = lane; i < m / 2; i += 32) {
                const int p = pr[i].x, q = pr[i].y;
                if (q < k && rot[4 * i + 1] != (R)0) {
                    A[q * k + p] = czero<C>();
                    A[p * k + q] = czero<C>();
                }
            }
            __syncwarp();
        }
        if (!__any_sync(0xffffffffu, nrw)) break;    // a sweep without a rotation: converged
    }
#undef JACOBI_COUNT_ROTATION
#undef JACOBI_MARK_ROUND
    for (int i = lane; i < k; i += 32) {
        const R di = jacobi_key(A[i * k + i].x);
        int pos = 0;
        for (int j = 0; j < k; ++j) {
            const R dj = jacobi_key(A[j * k + j].x);
            pos += (dj > di || (dj == di && j < i)) ? 1 : 0;
        }
        order[pos] = i;
    }
    __syncwarp();
    C* Vo = Vall + (long long)mat * k * k;
    for (int e = lane; e < k * k; e += 32) {
        const int col = e / k, row = e - col * k;
        Vo[e] = V[order[col] * k + row];
    }
}

// ---------------------------------------------------- Philox4x32-10 probes
__device__ __forceinline__ void philox10(uint32_t c[4], uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += W0; k1 += W1; }
        const uint32_t hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
        const uint32_t hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
}

template <typename C>
__global__ void k_gaussian(C* __restrict__ dst, int m, int k, long long sD, int batch, uint32_t k0, uint32_t k1,
                           const uint32_t* __restrict__ w2, const uint32_t* __restrict__ w3) {
    typedef decltype(dst->x) R;
    const long long per = (long long)m * k;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < per * batch; e += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(e / per);
        const long long r = e - b * per;
        const int j = (int)(r / m), i = (int)(r - (long long)j * m);
        uint32_t c[4] = {(uint32_t)(i >> 1), (uint32_t)j, w2[b], w3[b]};
        philox10(c, k0, k1);
        const uint32_t xa = (i & 1) ? c[2] : c[0], xb = (i & 1) ? c[3] : c[1];
        C v;
        if (sizeof(R) == 8) {
            const double u1 = ((double)xa + 1.0) * 2.3283064365386963e-10;
            const double u2 = (double)xb * 2.3283064365386963e-10;
            const double rho = sqrt(-log(u1));
            double s, cc;
            sincospi(2.0 * u2, &s, &cc);
            v.x = (R)(rho * cc);
            v.y = (R)(rho * s);
        } else {
            const float u1 = ((float)xa + 1.0f) * 2.3283064365386963e-10f;
            const float u2 = (float)xb * 2.3283064365386963e-10f;
            const float rho = sqrtf(-logf(u1));
            float s, cc;
            sincospif(2.0f * u2, &s, &cc);
            v.x = (R)(rho * cc);
            v.y = (R)(rho * s);
        }
        dst[b * sD + r] = v;
    }
}

// ------------------------------------------- blocked Gauss-Jordan inverse
// Panel step: the panel's nb columns (all n rows) are held in shared memory
// and reduced by Gauss-Jordan with partial pivoting over rows >= c.  The
// result is the panel of the block step
//     rows P:  A_PP^-1          rows R:  -A_RP A_PP^-1
// (after the row swaps), with the swaps recorded in piv.
template <typename C, int NT>
__global__ void __launch_bounds__(NT)
k_gj_panel(C* __restrict__ Aall, int n, long long sA, int k0, int nb, int* __restrict__ pivall) {
    typedef decltype(Aall->x) R;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    C* pan = reinterpret_cast<C*>(sm_raw);        // n x nb, column-major (ld n)
    __shared__ R rv[NT / 32];
    __shared__ int ri[NT / 32];
    __shared__ int pivrow;
    __shared__ C rowc[64];
    C* A = Aall + blockIdx.x * sA;
    int* piv = pivall + (long long)blockIdx.x * n;
    for (int e = threadIdx.x; e < n * nb; e += NT) {
        const int j = e / n, i = e - j * n;
        pan[e] = A[(long long)(k0 + j) * n + i];
    }
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        const int c = k0 + j;
        // argmax |pan[i][j]| over i >= c (first maximum wins)
        R best = -1;
        int bi = n;
        for (int i = c + threadIdx.x; i < n; i += NT) {
            const C v = pan[j * n + i];
            const R a = v.x * v.x + v.y * v.y;
            if (a > best || (a == best && i < bi)) { best = a; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const R ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if ((threadIdx.x & 31) == 0) { rv[threadIdx.x >> 5] = best; ri[threadIdx.x >> 5] = bi; }
        __syncthreads();
        if (threadIdx.x == 0) {
            R b2 = rv[0];
            int i2 = ri[0];
            for (int w = 1; w < NT / 32; ++w)
                if (rv[w] > b2 || (rv[w] == b2 && ri[w] < i2)) { b2 = rv[w]; i2 = ri[w]; }
            pivrow = i2 < n ? i2 : c;
            piv[c] = pivrow;
        }
        __syncthreads();
        const int p = pivrow;
        if (p != c)
            for (int t = threadIdx.x; t < nb; t += NT) {
                const C a = pan[t * n + c];
                pan[t * n + c] = pan[t * n + p];
                pan[t * n + p] = a;
            }
        __syncthreads();
        const C d = pan[j * n + c];
        const R den = d.x * d.x + d.y * d.y;
        const C inv = den > 0 ? mk(d.x / den, -d.y / den) : czero<C>();
        for (int t = threadIdx.x; t < nb; t += NT) rowc[t] = t == j ? inv : cmul(pan[t * n + c], inv);
        __syncthreads();
        // columns other than j first (they read column j), then column j and row c
        for (int e = threadIdx.x; e < n * nb; e += NT) {
            const int t = e / n, i = e - t * n;
            if (t == j || i == c) continue;
            pan[e] = csub(pan[e], cmul(pan[j * n + i], rowc[t]));
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += NT) {
            if (i == c) continue;
            const C f = pan[j * n + i];
            pan[j * n + i] = mk(-(f.x * inv.x - f.y * inv.y), -(f.x * inv.y + f.y * inv.x));
        }
        for (int t = threadIdx.x; t < nb; t += NT) pan[t * n + c] = rowc[t];
        __syncthreads();
    }
    for (int e = threadIdx.x; e < n * nb; e += NT) {
        const int j = e / n, i = e - j * n;
        A[(long long)(k0 + j) * n + i] = pan[e];
    }
}

// Register-resident panel step for n <= NT: thread i holds row i of the
// nb (<= 16) panel columns.  Each pivot step is an argmax over the rows at
// or below the pivot, a row exchange between two threads, and an update of
// every row by the scaled pivot row -- four barriers per column.
template <typename C, int NT, int NB>
__global__ void __launch_bounds__(NT)
k_gj_panel_reg(C* __restrict__ Aall, int n, long long sA, int k0, int nb, int* __restrict__ pivall,
               int* __restrict__ swlall) {
    typedef decltype(Aall->x) R;
    __shared__ R wbest[NT / 32];
    __shared__ int widx[NT / 32];
    __shared__ int pivrow;
    __shared__ int pvs[NB];
    __shared__ C rowc[NB];
    __shared__ C xbuf[2][NB];
    C* A = Aall + blockIdx.x * sA;
    int* piv = pivall + (long long)blockIdx.x * n;
    const int i = threadIdx.x;
    const bool own = i < n;
    C prow[NB];
#pragma unroll
    for (int t = 0; t < NB; ++t) prow[t] = (own && t < nb) ? A[(long long)(k0 + t) * n + i] : czero<C>();
    for (int j = 0; j < nb; ++j) {
        const int c = k0 + j;
        C pj = czero<C>();
#pragma unroll
        for (int t = 0; t < NB; ++t) if (t == j) pj = prow[t];
        R best = (own && i >= c) ? pj.x * pj.x + pj.y * pj.y : (R)-1;
        int bi = (own && i >= c) ? i : n;
        for (int o = 16; o > 0; o >>= 1) {
            const R ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if ((i & 31) == 0) { wbest[i >> 5] = best; widx[i >> 5] = bi; }
        __syncthreads();
        if (i < 32) {
            R b2 = i < NT / 32 ? wbest[i] : (R)-1;
            int i2 = i < NT / 32 ? widx[i] : n;
            for (int o = 16; o > 0; o >>= 1) {
                const R ob = __shfl_xor_sync(0xffffffffu, b2, o);
                const int oi = __shfl_xor_sync(0xffffffffu, i2, o);
                if (ob > b2 || (ob == b2 && oi < i2)) { b2 = ob; i2 = oi; }
            }
            if (i == 0) {
                pivrow = i2 < n ? i2 : c;
                piv[c] = pivrow;
                pvs[j] = pivrow;
            }
        }
        __syncthreads();
        const int p = pivrow;
        if (p != c) {
            if (i == c) {
#pragma unroll
                for (int t = 0; t < NB; ++t) xbuf[0][t] = prow[t];
            }
            if (i == p) {
#pragma unroll
                for (int t = 0; t < NB; ++t) xbuf[1][t] = prow[t];
            }
            __syncthreads();
            if (i == c) {
#pragma unroll
                for (int t = 0; t < NB; ++t) prow[t] = xbuf[1][t];
            }
            if (i == p) {
#pragma unroll
                for (int t = 0; t < NB; ++t) prow[t] = xbuf[0][t];
            }
        }
        if (i == c) {
            C d = czero<C>();
#pragma unroll
            for (int t = 0; t < NB; ++t) if (t == j) d = prow[t];
            const R den = d.x * d.x + d.y * d.y;
            const C inv = den > 0 ? mk(d.x / den, -d.y / den) : czero<C>();
#pragma unroll
            for (int t = 0; t < NB; ++t) {
                prow[t] = t == j ? inv : cmul(prow[t], inv);
                rowc[t] = prow[t];
            }
        }
        __syncthreads();
        if (own && i != c) {
            const C inv = rowc[j];
            C f = czero<C>();
#pragma unroll
            for (int t = 0; t < NB; ++t) if (t == j) f = prow[t];
#pragma unroll
            for (int t = 0; t < NB; ++t) {
                if (t == j) prow[t] = mk(-(f.x * inv.x - f.y * inv.y), -(f.x * inv.y + f.y * inv.x));
                else if (t < nb) prow[t] = csub(prow[t], cmul(f, rowc[t]));
            }
        }
    }
    if (own) {
#pragma unroll
        for (int t = 0; t < NB; ++t)
            if (t < nb) A[(long long)(k0 + t) * n + i] = prow[t];
    }
    // the panel's interchanges composed into one permutation sigma of the
    // positions they touch (count, then position/value pairs), for the update
    if (i == 0) {
        int* swl = swlall + (long long)blockIdx.x * (4 * NB + 1);
        int cnt = 0;
        for (int j = 0; j < nb; ++j) {
            const int c = k0 + j, p = pvs[j];
            if (p == c) continue;
            int ic = -1, ip = -1;
            for (int q = 0; q < cnt; ++q) {
                if (swl[1 + 2 * q] == c) ic = q;
                if (swl[1 + 2 * q] == p) ip = q;
            }
            if (ic < 0) { swl[1 + 2 * cnt] = c; swl[2 + 2 * cnt] = c; ic = cnt++; }
            if (ip < 0) { swl[1 + 2 * cnt] = p; swl[2 + 2 * cnt] = p; ip = cnt++; }
            const int t = swl[2 + 2 * ic]; swl[2 + 2 * ic] = swl[2 + 2 * ip]; swl[2 + 2 * ip] = t;
        }
        swl[0] = cnt;
    }
}

// Out-of-place block step for every column outside the panel, with the
// panel's row swaps folded into the reads:  row i of the result is
//   (i outside P) X[sigma(i)] + sum_t Pan[i][t] X[sigma(k0 + t)],
// sigma the composition of the swaps; panel columns are copied.
template <typename C>
__global__ void __launch_bounds__(256)
k_gj_update_oop(const C* __restrict__ Ain, C* __restrict__ Aout, int n, long long sA, int k0, int nb,
                const int* __restrict__ swlall, int swstride) {
    __shared__ C Ps[64][17];
    __shared__ C Xs[16][65];
    __shared__ int rmap[64];
    __shared__ int pmap[16];
    __shared__ int sw_pos[32], sw_val[32];
    __shared__ int nsw;
    const int b = blockIdx.z;
    const C* A = Ain + b * sA;
    C* O = Aout + b * sA;
    const int i0 = blockIdx.x * 64, j0 = blockIdx.y * 64;
    {
        // sigma on the positions the panel's swaps touch, composed by the panel kernel
        const int* swl = swlall + (long long)b * swstride;
        const int cnt = swl[0];
        if (threadIdx.x == 0) nsw = cnt;
        if (threadIdx.x < cnt) {
            sw_pos[threadIdx.x] = swl[1 + 2 * threadIdx.x];
            sw_val[threadIdx.x] = swl[2 + 2 * threadIdx.x];
        }
    }
    __syncthreads();
    auto sigma = [&](int pos) {
        for (int q = 0; q < nsw; ++q) if (sw_pos[q] == pos) return sw_val[q];
        return pos;
    };
    if (threadIdx.x < 64) rmap[threadIdx.x] = i0 + threadIdx.x < n ? sigma(i0 + threadIdx.x) : 0;
    if (threadIdx.x < 16) pmap[threadIdx.x] = threadIdx.x < nb ? sigma(k0 + threadIdx.x) : 0;
    __syncthreads();
    const int ty = threadIdx.x & 15, tx = threadIdx.x >> 4;   // consecutive lanes: consecutive rows
    // the old entries this thread's outputs add to, requested before the
    // panel product so that their latency overlaps it
    C aold[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int li = ty + 16 * p;
            const int gi = i0 + li, gj = j0 + tx + 16 * q;
            C v = czero<C>();
            if (gi < n && gj < n) {
                if (gj >= k0 && gj < k0 + nb) v = A[(long long)gj * n + gi];
                else if (!(gi >= k0 && gi < k0 + nb)) v = A[(long long)gj * n + rmap[li]];
            }
            aold[p][q] = v;
        }
    C acc[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = czero<C>();
    for (int e = threadIdx.x; e < 64 * 16; e += 256) {
        const int ii = e % 64, t = e / 64;
        const int gi = i0 + ii;
        Ps[ii][t] = (gi < n && t < nb) ? A[(long long)(k0 + t) * n + gi] : czero<C>();
        const int jj = e % 64;
        const int gj = j0 + jj;
        Xs[t][jj] = (gj < n && t < nb) ? A[(long long)gj * n + pmap[t]] : czero<C>();
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < 16; ++t) {
        C a[4], bb[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) { a[q] = Ps[ty + 16 * q][t]; bb[q] = Xs[t][tx + 16 * q]; }
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < 4; ++q) cfma(acc[p][q], a[p], bb[q]);
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int li = ty + 16 * p;
            const int gi = i0 + li, gj = j0 + tx + 16 * q;
            if (gi >= n || gj >= n) continue;
            C* o = O + (long long)gj * n + gi;
            if (gj >= k0 && gj < k0 + nb) *o = aold[p][q];
            else if (gi >= k0 && gi < k0 + nb) *o = acc[p][q];
            else *o = cadd(aold[p][q], acc[p][q]);
        }
}

// Apply the panel's swaps to every other column and copy its rows P aside.
template <typename C>
__global__ void k_gj_swap(C* __restrict__ Aall, int n, long long sA, int k0, int nb, const int* __restrict__ pivall,
                          C* __restrict__ XPall) {
    const int b = blockIdx.y;
    C* A = Aall + b * sA;
    const int* piv = pivall + (long long)b * n;
    C* XP = XPall + (long long)b * nb * n;
    for (int col = blockIdx.x * blockDim.x + threadIdx.x; col < n; col += gridDim.x * blockDim.x) {
        if (col >= k0 && col < k0 + nb) continue;
        C* a = A + (long long)col * n;
        for (int j = 0; j < nb; ++j) {
            const int c = k0 + j, p = piv[c];
            if (p != c) { const C t = a[c]; a[c] = a[p]; a[p] = t; }
        }
        for (int j = 0; j < nb; ++j) XP[(long long)col * nb + j] = a[k0 + j];
    }
}

// X_new = Pan * X_P + (rows outside P) X_old for every column outside P.
template <typename C>
__global__ void __launch_bounds__(256)
k_gj_update(C* __restrict__ Aall, int n, long long sA, int k0, int nb, const C* __restrict__ XPall) {
    __shared__ C Ps[64][17];
    __shared__ C Xs[16][65];
    const int b = blockIdx.z;
    C* A = Aall + b * sA;
    const C* XP = XPall + (long long)b * nb * n;
    const int i0 = blockIdx.x * 64, j0 = blockIdx.y * 64;
    const int ty = threadIdx.x & 15, tx = threadIdx.x >> 4;   // consecutive lanes: consecutive rows
    C acc[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = czero<C>();
    for (int t0 = 0; t0 < nb; t0 += 16) {
        for (int e = threadIdx.x; e < 64 * 16; e += 256) {
            const int i = e % 64, t = e / 64;
            const int gi = i0 + i;
            Ps[i][t] = (gi < n && t0 + t < nb) ? A[(long long)(k0 + t0 + t) * n + gi] : czero<C>();
            const int jj = e % 64, tt = e / 64;
            const int gj = j0 + jj;
            Xs[tt][jj] = (gj < n && t0 + tt < nb) ? XP[(long long)gj * nb + t0 + tt] : czero<C>();
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            C a[4], bb[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) { a[q] = Ps[ty + 16 * q][t]; bb[q] = Xs[t][tx + 16 * q]; }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) cfma(acc[p][q], a[p], bb[q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int gi = i0 + ty + 16 * p, gj = j0 + tx + 16 * q;
            if (gi >= n || gj >= n) continue;
            if (gj >= k0 && gj < k0 + nb) continue;
            C* a = A + (long long)gj * n + gi;
            if (gi >= k0 && gi < k0 + nb) *a = acc[p][q];
            else *a = cadd(*a, acc[p][q]);
        }
}

// Undo the row interchanges as column interchanges in reverse order.
template <typename C>
__global__ void k_gj_unscramble(C* __restrict__ Aall, int n, long long sA, const int* __restrict__ pivall) {
    const int b = blockIdx.y;
    C* A = Aall + b * sA;
    const int* piv = pivall + (long long)b * n;
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += gridDim.x * blockDim.x) {
        for (int c = n - 1; c >= 0; --c) {
            const int p = piv[c];
            if (p != c) {
                const C t = A[(long long)c * n + row];
                A[(long long)c * n + row] = A[(long long)p * n + row];
                A[(long long)p * n + row] = t;
            }
        }
    }
}

// ------------------------------------------------------------- norms
template <typename C>
__global__ void __launch_bounds__(256) k_norm_partial(const C* __restrict__ x, long long n, int nchunk, double* part) {
    const int b = blockIdx.y, ch = blockIdx.x;
    const long long per = (n + nchunk - 1) / nchunk;
    const long long r0 = ch * per, r1 = min(n, r0 + per);
    const C* xb = x + b * n;
    double s = 0;
    for (long long i = r0 + threadIdx.x; i < r1; i += 256) {
        const C v = xb[i];
        s += (double)v.x * v.x + (double)v.y * v.y;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int w = 0; w < 8; ++w) t += red[w];
        part[(long long)b * nchunk + ch] = t;
    }
}

__global__ void k_norm_reduce(const double* __restrict__ part, int nchunk, int batch, double* out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    double s = 0;
    for (int c = 0; c < nchunk; ++c) s += part[(long long)b * nchunk + c];
    out[b] = s;
}

template <typename C>
__global__ void k_cast64(const double2* __restrict__ s, C* __restrict__ d, long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        C v;
        v.x = s[e].x;
        v.y = s[e].y;
        d[e] = v;
    }
}

}  // namespace

// ================================================================ wrappers
template <typename CT>
size_t cn_small_smem(int m, int n) {
    const int ms = (m + 3) & ~3, ns = (n + 3) & ~3;
    const int G = std::max(1, 256 / ((ms / 4) * (ns / 4)));
    return sizeof(CT) * (32 * (size_t)(ms + ns + 2) + (size_t)G * m * n);
}

template <typename R>
lsw_status gemm(char opA, char opB, int m, int n, int k, typename Cx<R>::T alpha,
                const typename Cx<R>::T* A, int lda, long long sA,
                const typename Cx<R>::T* B, int ldb, long long sB,
                typename Cx<R>::T beta, typename Cx<R>::T* C, int ldc, long long sC,
                int batch, cudaStream_t st) {
    typedef typename Cx<R>::T CT;
    if (m <= 0 || n <= 0 || batch <= 0) return LSW_OK;
    const int oa = (opA == 'N' || opA == 'n') ? 0 : 1, ob = (opB == 'N' || opB == 'n') ? 0 : 1;
    if (k <= 0) {
        // C = beta C
        const CT zero = czero<CT>();
        k_gemm<CT, 64, 64><<<dim3((m + 63) / 64, (n + 63) / 64, batch), 256, 0, st>>>(
            oa, ob, m, n, 0, zero, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, 1, 0, nullptr);
        LSW_LAUNCH_CHECK();
        return LSW_OK;
    }
    // long inner products with a tiny result (Gram-Schmidt coefficients)
    if (oa == 1 && ob == 0 && n <= 4 && m * n <= 32 && k >= 128) {
        const long long want = std::max<long long>(1, 4864 / batch);
        const int kchunk = (int)std::max<long long>(512, ((k + want - 1) / want + 255) / 256 * 256);
        const int ksplit = (k + kchunk - 1) / kchunk;
        DevBuf part;
        LSW_TRY(part.alloc(sizeof(CT) * (size_t)ksplit * batch * m * n, st));
        const dim3 gr(ksplit, batch);
        switch (n) {
            case 1: k_gemm_cn_tiny<CT, 1><<<gr, 256, 0, st>>>(m, k, A, lda, sA, B, ldb, sB, kchunk, part.as<CT>(), batch); break;
            case 2: k_gemm_cn_tiny<CT, 2><<<gr, 256, 0, st>>>(m, k, A, lda, sA, B, ldb, sB, kchunk, part.as<CT>(), batch); break;
            case 3: k_gemm_cn_tiny<CT, 3><<<gr, 256, 0, st>>>(m, k, A, lda, sA, B, ldb, sB, kchunk, part.as<CT>(), batch); break;
            default: k_gemm_cn_tiny<CT, 4><<<gr, 256, 0, st>>>(m, k, A, lda, sA, B, ldb, sB, kchunk, part.as<CT>(), batch); break;
        }
        LSW_LAUNCH_CHECK();
        k_gemm_reduce<CT><<<grid_for((long long)batch * m * n), 256, 0, st>>>(m, n, batch, ksplit, part.as<CT>(), alpha,
                                                                              beta, C, ldc, sC);
        LSW_LAUNCH_CHECK();
        return LSW_OK;
    }
    // long inner products with a small result: split K, reduce in order
    if (oa == 1 && ob == 0 && m <= 64 && n <= 64 && (long long)m * n <= 4096 && k >= 128) {
        const long long want = std::max<long long>(1, 1216 / batch);
        const int kchunk = (int)std::max<long long>(256, ((k + want - 1) / want + 31) / 32 * 32);
        const int ksplit = (k + kchunk - 1) / kchunk;
        DevBuf part;
        LSW_TRY(part.alloc(sizeof(CT) * (size_t)ksplit * batch * m * n, st));
        static std::atomic<bool> attr_cn[2];
        if (!attr_cn[sizeof(R) == 8]) {
            LSW_CUDA(cudaFuncSetAttribute(k_gemm_cn_small<CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
            attr_cn[sizeof(R) == 8] = true;
        }
        k_gemm_cn_small<CT><<<dim3(ksplit, batch), 256, cn_small_smem<CT>(m, n), st>>>(m, n, k, A, lda, sA, B, ldb, sB, kchunk, part.as<CT>(),
                                                                   batch);
        LSW_LAUNCH_CHECK();
        k_gemm_reduce<CT><<<grid_for((long long)batch * m * n), 256, 0, st>>>(m, n, batch, ksplit, part.as<CT>(), alpha,
                                                                              beta, C, ldc, sC);
        LSW_LAUNCH_CHECK();
        return LSW_OK;
    }
    // tall times one column (the solvers' Krylov updates)
    if (oa == 0 && ob == 0 && k <= 64 && n == 1 && m >= 4096) {
        const long long pairs = ((long long)m + 1) / 2;
        k_gemv_tall<CT><<<dim3((unsigned)((pairs + 255) / 256), batch), 256, 0, st>>>(m, k, alpha, A, lda, sA, B, sB,
                                                                                      beta, C, sC);
        LSW_LAUNCH_CHECK();
        return LSW_OK;
    }
    // tall times small
    if (oa == 0 && ob == 0 && k <= 64 && n <= 64) {
        const int ngrp = (n + 15) / 16;
        const int rows_per = 256 / ngrp;
        static std::atomic<bool> attr_nn[2];
        if (!attr_nn[sizeof(R) == 8]) {
            LSW_CUDA(cudaFuncSetAttribute(k_gemm_nn_smallk<CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
            attr_nn[sizeof(R) == 8] = true;
        }
        k_gemm_nn_smallk<CT><<<dim3((m + rows_per - 1) / rows_per, batch), 256, sizeof(CT) * k * n, st>>>(
            m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC);
        LSW_LAUNCH_CHECK();
        return LSW_OK;
    }
    const bool narrow = n <= 32;
    const int BMv = narrow ? 128 : 64, BNv = narrow ? 32 : 64;
    const int gx = (m + BMv - 1) / BMv, gy = (n + BNv - 1) / BNv;
    auto launch = [&](int ks, int kc, CT* P) {
        if (narrow)
            k_gemm<CT, 128, 32><<<dim3(gx, gy, batch * ks), 256, 0, st>>>(oa, ob, m, n, k, alpha, A, lda, sA, B, ldb, sB,
                                                                           beta, C, ldc, sC, ks, kc, P);
        else
            k_gemm<CT, 64, 64><<<dim3(gx, gy, batch * ks), 256, 0, st>>>(oa, ob, m, n, k, alpha, A, lda, sA, B, ldb, sB,
                                                                          beta, C, ldc, sC, ks, kc, P);
    };
    // split K when the output grid alone cannot fill the GPU
    int ksplit = 1;
    const long long ctas = (long long)gx * gy * batch;
    if (ctas < 304 && k >= 256) {
        // chunks of at least 64: a few small outputs (the recompressions'
        // projections on the inversion's critical path) still fill the GPU
        ksplit = (int)std::min<long long>((608 + ctas - 1) / ctas, (k + 63) / 64);
        ksplit = std::max(1, std::min(ksplit, 64));
    }
    if (ksplit == 1) {
        launch(1, k, nullptr);
        LSW_LAUNCH_CHECK();
        return LSW_OK;
    }
    int kchunk = (k + ksplit - 1) / ksplit;
    kchunk = (kchunk + GBK - 1) / GBK * GBK;
    ksplit = (k + kchunk - 1) / kchunk;
    DevBuf part;
    LSW_TRY(part.alloc(sizeof(CT) * (size_t)ksplit * batch * m * n, st));
    launch(ksplit, kchunk, part.as<CT>());
    LSW_LAUNCH_CHECK();
    k_gemm_reduce<CT><<<grid_for((long long)batch * m * n), 256, 0, st>>>(m, n, batch, ksplit, part.as<CT>(), alpha,
                                                                          beta, C, ldc, sC);
    LSW_LAUNCH_CHECK();
    return LSW_OK;
}

template <typename R>
lsw_status qr_explicit(typename Cx<R>::T* A, int m, int k, long long sA, int batch, typename Cx<R>::T* work,
                       cudaStream_t st) {
    typedef typename Cx<R>::T CT;
    if (batch <= 0 || k <= 0 || m <= 0) return LSW_OK;
    if (k > 64) return LSW_ERR_INVALID_ARG;
    (void)work;
    // Two chunk shapes: 512 threads on up to ~200 KB of rows (one CTA per
    // SM), or 128 threads on <= 256 rows (three CTAs per SM).  The column
    // loop of a chunk is latency-bound, so small chunks are chosen whenever
    // the large ones would leave the GPU's 152 SMs short of three CTAs each.
    const size_t capL = 200 * 1024, capS = 72 * 1024;
    const int cmaxL = (int)std::min<size_t>(1024, (capL / sizeof(CT) - (size_t)k * k) / k);
    const int cmaxS = (int)std::min<size_t>(256, (capS / sizeof(CT) - (size_t)k * k) / k);
    static std::atomic<bool> attr[2];
    if (!attr[sizeof(R) == 8]) {
        LSW_CUDA(cudaFuncSetAttribute(k_tsqr_chunk<R, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)capL));
        LSW_CUDA(cudaFuncSetAttribute(k_tsqr_apply<R, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)capL));
        LSW_CUDA(cudaFuncSetAttribute(k_tsqr_chunk<R, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)capS));
        LSW_CUDA(cudaFuncSetAttribute(k_tsqr_apply<R, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)capS));
        attr[sizeof(R) == 8] = true;
    }
    const long long nchL = (m + cmaxL - 1) / cmaxL;
    // one large chunk per block (no second TSQR level) wins when the blocks
    // fit and there are no more of them than SMs
    const bool one_large = nchL == 1 && batch <= 152;
    const bool small = cmaxS >= 2 * k && (m <= cmaxS || (!one_large && nchL * batch < 3LL * 152));
    const int cmax = small ? cmaxS : cmaxL;
    // Tall-skinny QR (TSQR): factor row chunks independently, then the
    // stacked R factors, then combine.  Every chunk has >= cmax/2 >= k rows.
    const int nch = (m + cmax - 1) / cmax;
    const int rows = (m + nch - 1) / nch;
    const size_t smem = sizeof(CT) * ((size_t)rows * k + (size_t)k * k);
    auto chunk = [&](int nc, CT* S) {
        if (small) k_tsqr_chunk<R, 128><<<dim3(nc, batch), 128, smem, st>>>(A, m, k, sA, nc, S);
        else k_tsqr_chunk<R, 512><<<dim3(nc, batch), 512, smem, st>>>(A, m, k, sA, nc, S);
    };
    if (nch == 1) {
        DevBuf S;
        LSW_TRY(S.alloc(sizeof(CT) * (size_t)batch * k * k, st));
        KTimer kt("qr", st, sizeof(CT) * ((double)batch * m * k * 2 + (double)batch * k * k),
                  16.0 * batch * (double)m * k * k);
        chunk(1, S.as<CT>());
        LSW_LAUNCH_CHECK();
        return LSW_OK;
    }
    DevBuf S;
    const int ms = nch * k;
    LSW_TRY(S.alloc(sizeof(CT) * (size_t)batch * ms * k, st));
    {
        // reads and rewrites its rows, writes the R factors; Householder and
        // explicit Q: 16 m k^2 real flops per block (8 each)
        KTimer kt("qr", st, sizeof(CT) * ((double)batch * m * k * 2 + (double)batch * ms * k),
                  16.0 * batch * (double)m * k * k);
        chunk(nch, S.as<CT>());
        LSW_LAUNCH_CHECK();
    }
    LSW_TRY(qr_explicit<R>(S.as<CT>(), ms, k, (long long)ms * k, batch, nullptr, st));
    if (small) k_tsqr_apply<R, 128><<<dim3(nch, batch), 128, smem, st>>>(A, m, k, sA, nch, S.as<CT>());
    else k_tsqr_apply<R, 512><<<dim3(nch, batch), 512, smem, st>>>(A, m, k, sA, nch, S.as<CT>());
    LSW_LAUNCH_CHECK();
    return LSW_OK;
}

template <typename R>
lsw_status gram64(const typename Cx<R>::T* Y, int m, int k, long long sY, int batch, double2* G, cudaStream_t st) {
    typedef typename Cx<R>::T CT;
    if (batch <= 0 || k <= 0) return LSW_OK;
    // complex64 data: error-free products, FP64-accurate sums (small64.cu)
    if (sizeof(R) == 4) return gram64_c64(reinterpret_cast<const float2*>(Y), m, k, sY, batch, G, st);
    if (k > 64) return LSW_ERR_INVALID_ARG;   // 16 entries per thread at 256 threads
    const int nchunk = std::max(1, std::min((m + 255) / 256, std::max(1, 1216 / batch)));
    DevBuf part;
    LSW_TRY(part.alloc(sizeof(double2) * (size_t)batch * nchunk * k * k, st));
    k_gram_partial<CT><<<dim3(nchunk, batch), 256, sizeof(CT) * 33 * k, st>>>(Y, m, k, sY, nchunk,
                                                                                part.as<double2>());
    LSW_LAUNCH_CHECK();
    k_gram_reduce<<<grid_for((long long)batch * k * k), 256, 0, st>>>(part.as<double2>(), nchunk, k * k, batch, G);
    LSW_LAUNCH_CHECK();
    return LSW_OK;
}

template <typename R>
lsw_status heev_jacobi(const double2* G, typename Cx<R>::T* V, int k, int batch, cudaStream_t st, int polish) {
    typedef typename Cx<R>::T CT;
    if (batch <= 0 || k <= 0) return LSW_OK;
    if (k > 64) return LSW_ERR_INVALID_ARG;
    const int m = (k + 1) & ~1;
    const size_t per = sizeof(CT) * 2 * k * k + sizeof(R) * 4 * (m / 2) + sizeof(int2) * (m / 2) + sizeof(int) * 64;
    const size_t perA = (per + 15) & ~size_t(15);
    const int wpc = (int)std::max<size_t>(1, std::min<size_t>(8, (200 * 1024) / perA));
    static std::atomic<bool> attr[2];
    if (!attr[sizeof(R) == 8]) {
        LSW_CUDA(cudaFuncSetAttribute(k_heev_jacobi_warp<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        attr[sizeof(R) == 8] = true;
    }
    if (batch >= 4 * 152) {
        // many matrices: one warp each
        k_heev_jacobi_warp<R><<<(batch + wpc - 1) / wpc, 32 * wpc, perA * wpc, st>>>(G, V, k, batch, polish);
        LSW_LAUNCH_CHECK();
        return LSW_OK;
    }
    static std::atomic<bool> attrb[2];
    if (!attrb[sizeof(R) == 8]) {
        LSW_CUDA(cudaFuncSetAttribute(k_heev_jacobi<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
        attrb[sizeof(R) == 8] = true;
    }
    const size_t smb = sizeof(CT) * 3 * (size_t)k * k + sizeof(R) * 4 * (m / 2) + sizeof(int2) * (m / 2);
    // few matrices: the whole CTA of 1024 threads on each (a round is a
    // handful of dependent steps; more threads make each one shorter)
    k_heev_jacobi<R><<<batch, batch <= 2 * 152 ? 1024 : 256, smb, st>>>(G, V, k, polish);
    LSW_LAUNCH_CHECK();
    return LSW_OK;
}

template <typename R>
lsw_status cast_from64(const double2* src, typename Cx<R>::T* dst, long long n, cudaStream_t st) {
    k_cast64<typename Cx<R>::T><<<grid_for(n), 256, 0, st>>>(src, dst, n);
    LSW_LAUNCH_CHECK();
    return LSW_OK;
}

template <typename R>
lsw_status gaussian_fill(typename Cx<R>::T* dst, int m, int k, long long sD, int batch, uint64_t seed,
                         const uint32_t* w2, const uint32_t* w3, cudaStream_t st) {
    if (m <= 0 || k <= 0 || batch <= 0) return LSW_OK;
    k_gaussian<typename Cx<R>::T><<<grid_for((long long)m * k * batch), 256, 0, st>>>(
        dst, m, k, sD, batch, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32), w2, w3);
    LSW_LAUNCH_CHECK();
    return LSW_OK;
}

// Gauss-Jordan inverse of one small matrix (n <= GJS_MAX) per CTA, held in
// shared memory (column-major, leading dimension n + 1): for every column,
// pick the largest pivot below the diagonal, swap it up, scale its row and
// eliminate the column from every other row; the column swaps that undo the
// row interchanges come last.  Same pivoting as the blocked path.
template <typename C>
__global__ void __launch_bounds__(512)
k_gj_small(C* __restrict__ Aall, int n, long long sA) {
    typedef decltype(Aall->x) R;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int ld = n + 1;
    C* A = reinterpret_cast<C*>(sm_raw);              // n x ld
    C* rowj = A + (size_t)n * ld;                      // n
    C* colj = rowj + n;                                // n
    int* piv = reinterpret_cast<int*>(colj + n);       // n
    __shared__ R wbest[16];
    __shared__ int widx[16];
    __shared__ int pivrow;
    __shared__ C pval;
    C* G = Aall + blockIdx.x * sA;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int c = e / n, i = e - c * n;
        A[c * ld + i] = G[e];
    }
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        // pivot: largest |A(i, j)|, i >= j (lowest index on ties)
        R best = (R)-1;
        int bi = n;
        for (int i = j + threadIdx.x; i < n; i += blockDim.x) {
            const C a = A[j * ld + i];
            const R v = a.x * a.x + a.y * a.y;
            if (v > best) { best = v; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const R ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if ((threadIdx.x & 31) == 0) { wbest[threadIdx.x >> 5] = best; widx[threadIdx.x >> 5] = bi; }
        __syncthreads();
        if (threadIdx.x < 32) {
            const int nw = blockDim.x >> 5;
            R b2 = threadIdx.x < nw ? wbest[threadIdx.x] : (R)-1;
            int i2 = threadIdx.x < nw ? widx[threadIdx.x] : n;
            for (int o = 16; o > 0; o >>= 1) {
                const R ob = __shfl_xor_sync(0xffffffffu, b2, o);
                const int oi = __shfl_xor_sync(0xffffffffu, i2, o);
                if (ob > b2 || (ob == b2 && oi < i2)) { b2 = ob; i2 = oi; }
            }
            if (threadIdx.x == 0) {
                pivrow = i2 < n ? i2 : j;
                piv[j] = pivrow;
                pval = A[j * ld + pivrow];
            }
        }
        __syncthreads();
        const int p = pivrow;
        // swap rows j and p; keep the scaled pivot row and the old column j
        const C d = pval;
        const R den = d.x * d.x + d.y * d.y;
        const C inv = den > 0 ? mk(d.x / den, -d.y / den) : czero<C>();
        for (int c = threadIdx.x; c < n; c += blockDim.x) {
            const C aj = A[c * ld + j], ap = A[c * ld + p];
            A[c * ld + p] = aj;
            rowj[c] = c == j ? inv : cmul(ap, inv);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) colj[i] = i == j ? czero<C>() : A[j * ld + i];
        __syncthreads();
        // threads as 32 rows x 16 columns: lanes on consecutive rows, no division
        for (int c = threadIdx.x >> 5; c < n; c += 16) {
            const C rj = rowj[c];
            for (int i = threadIdx.x & 31; i < n; i += 32) {
                if (i == j) {
                    A[c * ld + i] = rj;
                } else {
                    const C f = colj[i];
                    A[c * ld + i] = c == j ? mk(-(f.x * rj.x - f.y * rj.y), -(f.x * rj.y + f.y * rj.x))
                                           : csub(A[c * ld + i], cmul(f, rj));
                }
            }
        }
        __syncthreads();
    }
    // undo the row interchanges as column interchanges, last first
    for (int j = n - 1; j >= 0; --j) {
        const int p = piv[j];
        if (p != j)
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const C t = A[j * ld + i];
                A[j * ld + i] = A[p * ld + i];
                A[p * ld + i] = t;
            }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int c = e / n, i = e - c * n;
        G[e] = A[c * ld + i];
    }
}

template <typename R>
lsw_status inverse_gj(typename Cx<R>::T* A, int n, long long sA, int batch, cudaStream_t st) {
    typedef typename Cx<R>::T CT;
    if (n <= 0 || batch <= 0) return LSW_OK;
    constexpr int NT = 1024;
    {
        // small matrices: one CTA each, entirely in shared memory
        const size_t smem = sizeof(CT) * ((size_t)n * (n + 1) + 2 * (size_t)n) + sizeof(int) * (size_t)n;
        if (n <= 160 && smem <= 200 * 1024) {
            static std::atomic<bool> attrs[2];
            if (!attrs[sizeof(R) == 8]) {
                LSW_CUDA(cudaFuncSetAttribute(k_gj_small<CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
                attrs[sizeof(R) == 8] = true;
            }
            k_gj_small<CT><<<batch, 512, smem, st>>>(A, n, sA);
            LSW_LAUNCH_CHECK();
            return LSW_OK;
        }
    }
    if (n <= NT) {
        // register panels + out-of-place updates, ping-pong between A and B
        constexpr int NB = sizeof(R) == 8 ? 8 : 16;
        const int nb = NB;
        DevBuf piv, B, swl;
        LSW_TRY(piv.alloc(sizeof(int) * (size_t)n * batch, st));
        LSW_TRY(B.alloc(sizeof(CT) * (size_t)sA * batch, st));
        const int swstride = 4 * NB + 1;
        LSW_TRY(swl.alloc(sizeof(int) * (size_t)swstride * batch, st));
        CT* cur = A;
        CT* nxt = B.as<CT>();
        for (int k0 = 0; k0 < n; k0 += nb) {
            const int w = std::min(nb, n - k0);
            k_gj_panel_reg<CT, NT, NB><<<batch, NT, 0, st>>>(cur, n, sA, k0, w, piv.as<int>(), swl.as<int>());
            LSW_LAUNCH_CHECK();
            if (w == n) continue;
            {
                // reads and writes every matrix once; 8 n^2 w real flops each
                KTimer kt("gj_update", st, 2.0 * sizeof(CT) * (double)n * n * batch, 8.0 * (double)n * n * w * batch);
                k_gj_update_oop<CT><<<dim3((n + 63) / 64, (n + 63) / 64, batch), 256, 0, st>>>(cur, nxt, n, sA, k0, w,
                                                                                              swl.as<int>(), swstride);
                LSW_LAUNCH_CHECK();
            }
            std::swap(cur, nxt);
        }
        if (cur != A) {
            LSW_CUDA(cudaMemcpy2DAsync(A, sizeof(CT) * sA, cur, sizeof(CT) * sA, sizeof(CT) * (size_t)n * n, batch,
                                       cudaMemcpyDeviceToDevice, st));
        }
        k_gj_unscramble<CT><<<dim3((n + 255) / 256, batch), 256, 0, st>>>(A, n, sA, piv.as<int>());
        LSW_LAUNCH_CHECK();
        return LSW_OK;
    }
    const size_t cap = 200 * 1024;
    int nb = 16;
    while (nb > 1 && (size_t)n * nb * sizeof(CT) > cap) nb >>= 1;
    if ((size_t)n * nb * sizeof(CT) > cap) return LSW_ERR_UNSUPPORTED_SIZE;
    static std::atomic<bool> attr{false};
    if (!attr) {
        LSW_CUDA(cudaFuncSetAttribute(k_gj_panel<CT, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap));
        attr = true;
    }
    DevBuf piv, xp;
    LSW_TRY(piv.alloc(sizeof(int) * (size_t)n * batch, st));
    LSW_TRY(xp.alloc(sizeof(CT) * (size_t)nb * n * batch, st));
    for (int k0 = 0; k0 < n; k0 += nb) {
        const int w = std::min(nb, n - k0);
        k_gj_panel<CT, NT><<<batch, NT, sizeof(CT) * (size_t)n * w, st>>>(A, n, sA, k0, w, piv.as<int>());
        LSW_LAUNCH_CHECK();
        if (w == n) continue;
        k_gj_swap<CT><<<dim3((n + 255) / 256, batch), 256, 0, st>>>(A, n, sA, k0, w, piv.as<int>(), xp.as<CT>());
        LSW_LAUNCH_CHECK();
        k_gj_update<CT><<<dim3((n + 63) / 64, (n + 63) / 64, batch), 256, 0, st>>>(A, n, sA, k0, w, xp.as<CT>());
        LSW_LAUNCH_CHECK();
    }
    k_gj_unscramble<CT><<<dim3((n + 255) / 256, batch), 256, 0, st>>>(A, n, sA, piv.as<int>());
    LSW_LAUNCH_CHECK();
    return LSW_OK;
}

template <typename R>
lsw_status norms2(const typename Cx<R>::T* x, long long n, int batch, double* out, cudaStream_t st) {
    if (batch <= 0) return LSW_OK;
    const int nchunk = (int)std::max<long long>(1, std::min<long long>((n + 4095) / 4096, std::max(1, 1216 / batch)));
    DevBuf part;
    LSW_TRY(part.alloc(sizeof(double) * (size_t)nchunk * batch, st));
    k_norm_partial<typename Cx<R>::T><<<dim3(nchunk, batch), 256, 0, st>>>(x, n, nchunk, part.as<double>());
    LSW_LAUNCH_CHECK();
    k_norm_reduce<<<(batch + 255) / 256, 256, 0, st>>>(part.as<double>(), nchunk, batch, out);
    LSW_LAUNCH_CHECK();
    return LSW_OK;
}

#define LSW_INST(R)                                                                                               \
    template lsw_status gemm<R>(char, char, int, int, int, Cx<R>::T, const Cx<R>::T*, int, long long,             \
                                const Cx<R>::T*, int, long long, Cx<R>::T, Cx<R>::T*, int, long long, int,        \
                                cudaStream_t);                                                                    \
    template lsw_status qr_explicit<R>(Cx<R>::T*, int, int, long long, int, Cx<R>::T*, cudaStream_t);             \
    template lsw_status gram64<R>(const Cx<R>::T*, int, int, long long, int, double2*, cudaStream_t);             \
    template lsw_status heev_jacobi<R>(const double2*, Cx<R>::T*, int, int, cudaStream_t, int);                        \
    template lsw_status cast_from64<R>(const double2*, Cx<R>::T*, long long, cudaStream_t);                        \
    template lsw_status gaussian_fill<R>(Cx<R>::T*, int, int, long long, int, uint64_t, const uint32_t*,          \
                                         const uint32_t*, cudaStream_t);                                          \
    template lsw_status inverse_gj<R>(Cx<R>::T*, int, long long, int, cudaStream_t);                              \
    template lsw_status norms2<R>(const Cx<R>::T*, long long, int, double*, cudaStream_t);
LSW_INST(float)
LSW_INST(double)
#undef LSW_INST

}  // namespace lsw
