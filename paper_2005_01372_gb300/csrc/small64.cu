// FP64 arithmetic of the randomized sketches (Algorithm 1/2): the Gram
// matrices of sketch blocks, the thin QR of the complex64 sketches by
// shifted Cholesky QR, and the Hermitian eigen-decomposition of the small
// Gram matrix that truncates Q Yt^H to rank r.  The tall factors (Y, Q, Yt)
// stay in the working precision; every k x k matrix derived from them
// (k <= 64 columns) is formed and factored in FP64.
//
// FP64 on this GPU runs at 1/62 of the FP32 rate (1.25 against 78 TFLOP/s,
// measured), so the Gram of a complex64 block is accumulated with
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

constexpr int GT_ROWS = 32;   // rows per tile (one compensated sum)
constexpr int GT_MAXQ = 9;    // pairs per thread: 256 * 9 >= 64 * 65 / 2

// Partial Gram of rows [r0, r1) of block b: part[(b * nchunk + ch) * npair + p]
// for the upper-triangle pairs p.  Columns are staged in shared memory in
// tiles of 32 rows (odd stride: the lanes of a warp read different banks).
__global__ void __launch_bounds__(256)
k_gram_c64(const float2* __restrict__ Y, int m, int k, long long sY, int nchunk, double2* __restrict__ part) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    float2* sy = reinterpret_cast<float2*>(sm_raw);   // k columns x (GT_ROWS + 1)
    const int b = blockIdx.y, ch = blockIdx.x;
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
        double2 s = make_double2(0.0, 0.0);
        for (int c = 0; c < nchunk; ++c) {
            const double2 v = part[((long long)b * nchunk + c) * npair + p];
            s.x += v.x;
            s.y += v.y;
        }
        if (i > j) s.y = -s.y;   // G(i, j) = conj(G(j, i))
        G[e] = s;
    }
}

// ------------------------------------------- Cholesky and R^-1 (FP64)
// One warp per matrix: G + shift I = L L^H (L = R^H lower triangular), then
// X = L^-1 by forward substitution (each lane owns columns of X), and
// Rinv = R^-1 = X^H.  A non-positive pivot restarts the factorisation with a
// larger shift (1e-15 tr(G) / k, then x100, at most 12 times).  A block with
// tr(G) = 0 gets Rinv = 0 (its Q is zero, which the truncation keeps as a
// zero block).
template <typename C>
__global__ void __launch_bounds__(128)
k_chol_rinv(const double2* __restrict__ Gall, int k, int batch, double shift_rel, C* __restrict__ Rall) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mat = blockIdx.x * (blockDim.x >> 5) + w;
    if (mat >= batch) return;
    const int ld = k + 1;
    double2* L = reinterpret_cast<double2*>(sm_raw) + (size_t)w * 2 * k * ld;
    double2* X = L + (size_t)k * ld;
    const double2* G = Gall + (long long)mat * k * k;
    C* Rout = Rall + (long long)mat * k * k;
    double tr = 0.0;
    for (int i = 0; i < k; ++i) tr += G[i * k + i].x;
    tr /= k;
    if (!(tr > 0.0) || !isfinite(tr)) {
        const double fill = (tr == 0.0) ? 0.0 : NAN;
        for (int e = lane; e < k * k; e += 32) { Rout[e].x = fill; Rout[e].y = fill; }
        return;
    }
    double shift = shift_rel * tr;
    bool ok = false;
    for (int attempt = 0; attempt < 13 && !ok; ++attempt) {
        for (int e = lane; e < k * k; e += 32) {
            const int j = e / k, i = e - j * k;
            double2 v = G[e];
            if (i == j) { v.x += shift; v.y = 0.0; }
            L[j * ld + i] = v;
        }
        __syncwarp();
        ok = true;
        for (int j = 0; j < k; ++j) {
            const double djj = L[j * ld + j].x;
            if (!(djj > 0.0) || !isfinite(djj)) { ok = false; break; }
            const double rjj = sqrt(djj), irj = 1.0 / rjj;
            __syncwarp();
            for (int i = j + 1 + lane; i < k; i += 32) {
                double2 v = L[j * ld + i];
                L[j * ld + i] = make_double2(v.x * irj, v.y * irj);
            }
            if (lane == 0) L[j * ld + j] = make_double2(rjj, 0.0);
            __syncwarp();
            // trailing lower triangle: L(i, l) -= L(i, j) conj(L(l, j)), j < l <= i
            const int nt = k - 1 - j;
            for (int e = lane; e < nt * nt; e += 32) {
                const int l = j + 1 + e / nt, i = j + 1 + e % nt;
                if (i < l) continue;
                const double2 a = L[j * ld + i], bq = L[j * ld + l];
                double2 v = L[l * ld + i];
                v.x -= a.x * bq.x + a.y * bq.y;
                v.y -= a.y * bq.x - a.x * bq.y;
                L[l * ld + i] = v;
            }
            __syncwarp();
        }
        __syncwarp();
        if (!ok) shift = shift > 0.0 ? shift * 100.0 : 1e-15 * tr;
    }
    if (!ok) {
        for (int e = lane; e < k * k; e += 32) { Rout[e].x = NAN; Rout[e].y = NAN; }
        return;
    }
    // X = L^-1 (lower): column c by forward substitution
    for (int c = lane; c < k; c += 32) {
        for (int i = 0; i < c; ++i) X[c * ld + i] = make_double2(0.0, 0.0);
        X[c * ld + c] = make_double2(1.0 / L[c * ld + c].x, 0.0);
        for (int i = c + 1; i < k; ++i) {
            double sx = 0.0, sy = 0.0;
            for (int t = c; t < i; ++t) {
                const double2 a = L[t * ld + i], x = X[c * ld + t];
                sx += a.x * x.x - a.y * x.y;
                sy += a.x * x.y + a.y * x.x;
            }
            const double il = 1.0 / L[i * ld + i].x;
            X[c * ld + i] = make_double2(-sx * il, -sy * il);
        }
    }
    __syncwarp();
    // Rinv(i, j) = conj(X(j, i)), upper triangular
    for (int e = lane; e < k * k; e += 32) {
        const int j = e / k, i = e - j * k;
        C v;
        if (i <= j) {
            const double2 x = X[i * ld + j];
            v.x = x.x;
            v.y = -x.y;
        } else {
            v.x = 0;
            v.y = 0;
        }
        Rout[e] = v;
    }
}

// ------------------------------------ Hermitian eigen-decomposition (FP64)
// One warp per matrix (k <= 64).  (1) Householder reduction to a real
// symmetric tridiagonal T = Q^H A Q, Q = H_0 ... H_{k-2}, each
// H_j = I - tau_j v_j v_j^H chosen so that H_j^H maps the column below the
// diagonal onto a real multiple of e_1 (the reflector convention of LAPACK's
// zlarfg); the two-sided update is A <- A - v w^H - w v^H with p = tau A v,
// w = p - (s / 2) v, s = conj(tau) v^H p (real).  (2) Implicit QL iteration
// with Wilkinson shifts on T (Bowdler, Martin, Reinsch and Wilkinson, Numer.
// Math. 11, 1968): lane 0 runs the scalar recurrence of one sweep and
// records its plane rotations, then every lane applies them to its rows of
// the eigenvector matrix.  (3) V = H_0 ... H_{k-2} Z, one column per lane.
// Output: the eigenvectors as columns, by decreasing eigenvalue.  An
// eigenvalue that needs more than 60 QL sweeps marks the result NaN.
struct QlWarp {
    double2* A;      // k x ld: the matrix, then the reflectors v_j below the diagonal
    double2* V;      // k x ld: Z (real parts), then the eigenvectors
    double* d;       // k
    double* e;       // k
    double* rc;      // 64: rotation cosines of one sweep
    double* rs;      // 64: rotation sines
    double2* tau;    // k
    double2* wv;     // 64
    int* order;      // 64
};

__host__ __device__ inline size_t ql_warp_bytes(int k) {
    const size_t ld = (size_t)k + 1;
    return sizeof(double2) * (2 * (size_t)k * ld + (size_t)k + 64) + sizeof(double) * (2 * (size_t)k + 128) +
           sizeof(int) * 64 + 16;
}

template <typename C>
__global__ void __launch_bounds__(64)
k_heev_ql(const double2* __restrict__ Gall, C* __restrict__ Vall, int k, int batch) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mat = blockIdx.x * (blockDim.x >> 5) + w;
    if (mat >= batch) return;
    const int ld = k + 1;
    const size_t per = (ql_warp_bytes(k) + 15) & ~size_t(15);
    unsigned char* base = sm_raw + (size_t)w * per;
    QlWarp s;
    s.A = reinterpret_cast<double2*>(base);
    s.V = s.A + (size_t)k * ld;
    s.tau = s.V + (size_t)k * ld;
    s.wv = s.tau + k;
    s.d = reinterpret_cast<double*>(s.wv + 64);
    s.e = s.d + k;
    s.rc = s.e + k;
    s.rs = s.rc + 64;
    s.order = reinterpret_cast<int*>(s.rs + 64);
    const double2* G = Gall + (long long)mat * k * k;
    for (int q = lane; q < k * k; q += 32) {
        const int j = q / k, i = q - j * k;
        s.A[j * ld + i] = G[q];
        s.V[j * ld + i] = make_double2(i == j ? 1.0 : 0.0, 0.0);
    }
    __syncwarp();
    // (1) tridiagonalisation
    for (int j = 0; j + 1 < k; ++j) {
        const int m = k - 1 - j;                      // rows j+1 .. k-1
        double2* x = s.A + j * ld + j + 1;            // column j below the diagonal
        double part = 0.0;
        for (int i = 1 + lane; i < m; i += 32) part += x[i].x * x[i].x + x[i].y * x[i].y;
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        const double2 alpha = x[0];
        double2 t = make_double2(0.0, 0.0);
        double beta = alpha.x;
        if (part > 0.0 || alpha.y != 0.0) {
            const double nrm = sqrt(alpha.x * alpha.x + alpha.y * alpha.y + part);
            beta = alpha.x >= 0.0 ? -nrm : nrm;
            t = make_double2((beta - alpha.x) / beta, -alpha.y / beta);
            // v = [1; x[1:] / (alpha - beta)]
            const double dr = alpha.x - beta, di = alpha.y;
            const double den = dr * dr + di * di;
            const double ir = dr / den, ii = -di / den;
            __syncwarp();
            for (int i = 1 + lane; i < m; i += 32) {
                const double2 v = x[i];
                x[i] = make_double2(v.x * ir - v.y * ii, v.x * ii + v.y * ir);
            }
            if (lane == 0) x[0] = make_double2(1.0, 0.0);
            __syncwarp();
            // p = tau A22 v, rows lane and lane + 32 (m <= 63)
            double2 p[2];
            for (int u = 0; u < 2; ++u) {
                const int i = lane + 32 * u;
                double sx = 0.0, sy = 0.0;
                if (i < m) {
                    for (int l = 0; l < m; ++l) {
                        const double2 a = s.A[(j + 1 + l) * ld + j + 1 + i], v = x[l];
                        sx += a.x * v.x - a.y * v.y;
                        sy += a.x * v.y + a.y * v.x;
                    }
                }
                p[u] = make_double2(t.x * sx - t.y * sy, t.x * sy + t.y * sx);
            }
            // c = v^H p, s = Re(conj(tau) c)
            double cx = 0.0, cy = 0.0;
            for (int u = 0; u < 2; ++u) {
                const int i = lane + 32 * u;
                if (i < m) {
                    const double2 v = x[i];
                    cx += v.x * p[u].x + v.y * p[u].y;
                    cy += v.x * p[u].y - v.y * p[u].x;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                cx += __shfl_xor_sync(0xffffffffu, cx, o);
                cy += __shfl_xor_sync(0xffffffffu, cy, o);
            }
            const double sr = t.x * cx + t.y * cy;
            for (int u = 0; u < 2; ++u) {
                const int i = lane + 32 * u;
                if (i < m) {
                    const double2 v = x[i];
                    s.wv[i] = make_double2(p[u].x - 0.5 * sr * v.x, p[u].y - 0.5 * sr * v.y);
                }
            }
            __syncwarp();
            // A22 -= v w^H + w v^H
            for (int q = lane; q < m * m; q += 32) {
                const int l = q / m, i = q - l * m;
                const double2 vi = x[i], vl = x[l], wi = s.wv[i], wl = s.wv[l];
                double2 a = s.A[(j + 1 + l) * ld + j + 1 + i];
                a.x -= vi.x * wl.x + vi.y * wl.y + wi.x * vl.x + wi.y * vl.y;
                a.y -= vi.y * wl.x - vi.x * wl.y + wi.y * vl.x - wi.x * vl.y;
                s.A[(j + 1 + l) * ld + j + 1 + i] = a;
            }
            __syncwarp();
        }
        if (lane == 0) {
            s.tau[j] = t;
            s.e[j] = beta;
            s.d[j] = s.A[j * ld + j].x;
        }
        __syncwarp();
    }
    if (lane == 0) {
        s.d[k - 1] = s.A[(k - 1) * ld + k - 1].x;
        s.e[k - 1] = 0.0;
        s.tau[k - 1] = make_double2(0.0, 0.0);
    }
    __syncwarp();
    // (2) implicit QL
    int failed = 0;
    for (int l = 0; l < k && !failed; ++l) {
        for (int iter = 0;; ++iter) {
            // lane 0: one sweep; code: 0 converged, 1 rotations in rc/rs for
            // i = m-1 down to lo, 2 failed
            int code = 0, mm = l, lo = l;
            if (lane == 0) {
                double* d = s.d;
                double* e = s.e;
                int m = l;
                for (; m < k - 1; ++m) {
                    const double dd = fabs(d[m]) + fabs(d[m + 1]);
                    if (fabs(e[m]) <= DBL_EPSILON * dd) break;
                }
                mm = m;
                if (m == l) code = 0;
                else if (iter == 60) code = 2;
                else {
                    code = 1;
                    double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
                    double r = hypot(g, 1.0);
                    g = d[m] - d[l] + e[l] / (g + (g >= 0.0 ? r : -r));
                    double sn = 1.0, cs = 1.0, p = 0.0;
                    int i = m - 1;
                    bool under = false;
                    for (; i >= l; --i) {
                        const double f = sn * e[i], b = cs * e[i];
                        r = hypot(f, g);
                        e[i + 1] = r;
                        if (r == 0.0) {
                            d[i + 1] -= p;
                            e[m] = 0.0;
                            under = true;
                            break;
                        }
                        sn = f / r;
                        cs = g / r;
                        g = d[i + 1] - p;
                        r = (d[i] - g) * sn + 2.0 * cs * b;
                        p = sn * r;
                        d[i + 1] = g + p;
                        g = cs * r - b;
                        s.rc[i] = cs;
                        s.rs[i] = sn;
                    }
                    lo = under ? i + 1 : l;
                    if (!under) {
                        d[l] -= p;
                        e[l] = g;
                        e[m] = 0.0;
                    }
                }
            }
            code = __shfl_sync(0xffffffffu, code, 0);
            mm = __shfl_sync(0xffffffffu, mm, 0);
            lo = __shfl_sync(0xffffffffu, lo, 0);
            __syncwarp();
            if (code == 0) break;
            if (code == 2) { failed = 1; break; }
            for (int i = mm - 1; i >= lo; --i) {
                const double cs = s.rc[i], sn = s.rs[i];
                for (int row = lane; row < k; row += 32) {
                    const double zf = s.V[(i + 1) * ld + row].x, zi = s.V[i * ld + row].x;
                    s.V[(i + 1) * ld + row].x = sn * zi + cs * zf;
                    s.V[i * ld + row].x = cs * zi - sn * zf;
                }
            }
            __syncwarp();
        }
    }
    __syncwarp();
    // (3) V = H_0 ... H_{k-2} Z, column by column
    for (int col = lane; col < k; col += 32) {
        double2* vc = s.V + col * ld;
        for (int j = k - 2; j >= 0; --j) {
            const double2 t = s.tau[j];
            if (t.x == 0.0 && t.y == 0.0) continue;
            const double2* v = s.A + j * ld + j + 1;    // rows j+1 .. k-1, v[0] = 1
            double sx = 0.0, sy = 0.0;
            for (int i = j + 1; i < k; ++i) {
                const double2 vv = v[i - j - 1], x = vc[i];
                sx += vv.x * x.x + vv.y * x.y;
                sy += vv.x * x.y - vv.y * x.x;
            }
            const double tx = t.x * sx - t.y * sy, ty = t.x * sy + t.y * sx;
            for (int i = j + 1; i < k; ++i) {
                const double2 vv = v[i - j - 1];
                vc[i].x -= vv.x * tx - vv.y * ty;
                vc[i].y -= vv.x * ty + vv.y * tx;
            }
        }
    }
    if (lane == 0) {
        for (int i = 0; i < k; ++i) s.order[i] = i;
        for (int i = 0; i < k; ++i) {
            int best = i;
            for (int jj = i + 1; jj < k; ++jj)
                if (s.d[s.order[jj]] > s.d[s.order[best]]) best = jj;
            const int tmp = s.order[i];
            s.order[i] = s.order[best];
            s.order[best] = tmp;
        }
    }
    __syncwarp();
    C* Vo = Vall + (long long)mat * k * k;
    for (int q = lane; q < k * k; q += 32) {
        const int col = q / k, row = q - col * k;
        const double2 v = s.V[s.order[col] * ld + row];
        C o;
        o.x = failed ? NAN : v.x;
        o.y = failed ? NAN : v.y;
        Vo[q] = o;
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

lsw_status gram64_c64(const float2* Y, int m, int k, long long sY, int batch, double2* G, cudaStream_t st) {
    if (batch <= 0 || k <= 0) return LSW_OK;
    if (k > 64) return LSW_ERR_INVALID_ARG;
    const int nchunk = std::max(1, std::min((m + 255) / 256, std::max(1, 1216 / batch)));
    const int npair = k * (k + 1) / 2;
    DevBuf part;
    LSW_TRY(part.alloc(sizeof(double2) * (size_t)batch * nchunk * npair, st));
    k_gram_c64<<<dim3(nchunk, batch), 256, sizeof(float2) * (GT_ROWS + 1) * k, st>>>(Y, m, k, sY, nchunk,
                                                                                        part.as<double2>());
    LSW_LAUNCH_CHECK();
    k_gram_c64_reduce<<<grid_small((long long)batch * k * k), 256, 0, st>>>(part.as<double2>(), nchunk, k, batch, G);
    LSW_LAUNCH_CHECK();
    return LSW_OK;
}

template <typename R>
lsw_status chol_rinv(const double2* G, int k, int batch, double shift_rel, typename Cx<R>::T* Rinv, cudaStream_t st) {
    typedef typename Cx<R>::T C;
    if (batch <= 0 || k <= 0) return LSW_OK;
    if (k > 64) return LSW_ERR_INVALID_ARG;
    const size_t per = sizeof(double2) * 2 * (size_t)k * (k + 1);
    const int wpc = (int)std::max<size_t>(1, std::min<size_t>(4, (160 * 1024) / per));
    static std::atomic<bool> attr{false};
    if (!attr.load()) {
        LSW_CUDA(cudaFuncSetAttribute(k_chol_rinv<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        attr.store(true);
    }
    k_chol_rinv<C><<<(batch + wpc - 1) / wpc, 32 * wpc, per * wpc, st>>>(G, k, batch, shift_rel, Rinv);
    LSW_LAUNCH_CHECK();
    return LSW_OK;
}

template <typename R>
lsw_status heev_ql(const double2* G, typename Cx<R>::T* V, int k, int batch, cudaStream_t st) {
    typedef typename Cx<R>::T C;
    if (batch <= 0 || k <= 0) return LSW_OK;
    if (k > 64) return LSW_ERR_INVALID_ARG;
    const size_t perA = (ql_warp_bytes(k) + 15) & ~size_t(15);
    const int wpc = (int)std::max<size_t>(1, std::min<size_t>(2, (200 * 1024) / perA));
    static std::atomic<bool> attr{false};
    if (!attr.load()) {
        LSW_CUDA(cudaFuncSetAttribute(k_heev_ql<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024));
        attr.store(true);
    }
    k_heev_ql<C><<<(batch + wpc - 1) / wpc, 32 * wpc, perA * wpc, st>>>(G, V, k, batch);
    LSW_LAUNCH_CHECK();
    return LSW_OK;
}

// Thin QR of complex64 sketch blocks, Q returned in place of A (m x k, ld m,
// block stride sA).  Tall blocks (m >= 4k): shifted Cholesky QR3 (Fukaya,
// Nakatsukasa, Yanagisawa, Yamamoto, SIAM J. Sci. Comput. 42, 2020): one pass
// on G + s I with s = 1e-13 tr(G) / k, then two plain passes, each an FP64
// Gram, an FP64 Cholesky factor and a product with R^-1 in the data's
// precision.  Short blocks: Householder QR in FP64 on an upcast copy.
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
    KTimer kt("qr", st, 8.0 * batch * (double)mk * 7, 3.0 * batch * (8.0 * m * k * (k + 1) / 2 * 5 + 8.0 * m * k * k / 2));
    DevBuf G, Ri, W;
    LSW_TRY(G.alloc(sizeof(double2) * (size_t)batch * k * k, st));
    LSW_TRY(Ri.alloc(sizeof(float2) * (size_t)batch * k * k, st));
    LSW_TRY(W.alloc(sizeof(float2) * (size_t)mk * batch, st));
    const float2 one = make_float2(1.f, 0.f), zero = make_float2(0.f, 0.f);
    auto pass = [&](const float2* src, long long ss, float2* dst, long long sd, double shift) -> lsw_status {
        LSW_TRY(gram64_c64(src, m, k, ss, batch, G.as<double2>(), st));
        LSW_TRY(chol_rinv<float>(G.as<double2>(), k, batch, shift, Ri.as<float2>(), st));
        return gemm<float>('N', 'N', m, k, k, one, src, m, ss, Ri.as<float2>(), k, (long long)k * k, zero, dst, m, sd,
                           batch, st);
    };
    LSW_TRY(pass(A, sA, W.as<float2>(), mk, 1e-13));
    LSW_TRY(pass(W.as<float2>(), mk, A, sA, 0.0));
    LSW_TRY(pass(A, sA, W.as<float2>(), mk, 0.0));
    LSW_CUDA(cudaMemcpy2DAsync(A, sizeof(float2) * (size_t)sA, W.p, sizeof(float2) * (size_t)mk,
                               sizeof(float2) * (size_t)mk, batch, cudaMemcpyDeviceToDevice, st));
    return LSW_OK;
}

template lsw_status chol_rinv<float>(const double2*, int, int, double, float2*, cudaStream_t);
template lsw_status chol_rinv<double>(const double2*, int, int, double, double2*, cudaStream_t);
template lsw_status heev_ql<float>(const double2*, float2*, int, int, cudaStream_t);
template lsw_status heev_ql<double>(const double2*, double2*, int, int, cudaStream_t);

}  // namespace lsw
