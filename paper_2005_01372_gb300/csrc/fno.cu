// Fourier neural operator used as a learned right preconditioner: forward,
// backward (G = dL/dRe + i dL/dIm convention), Adam, and the preconditioner
// apply, all in FP32 complex on the library's batched GEMMs.
//
// Network (complex): v = P x + p;  v <- sigma(K_l v + W_l v + b_l) for
// l < L (no sigma on the last layer);  y = x0 + Q v + q.  K_l keeps the 2m x 2m
// modes kz, kx in {0..m-1} U {n-m..n-1} of the 2D DFT and mixes channels per
// mode with R_l[mode] (W x W).  sigma: GELU on real and imaginary parts.
// The output adds the input's residual channel x0: y = x0 + Q v + q.
//
// Layouts.  A field is nz x nx, strip order; a batch of samples holds W
// fields per sample, sample after sample, so sample b is the column-major
// n x W matrix V_b.  Parameters live in one buffer in this order (all
// column-major complex): P^T (2 x W), p (W), then per layer R (4m^2 modes,
// each W_out x W_in), W^T (W x W), b (W), then Q^T (W x 1), q (1).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <new>
#include <vector>

#include "lsw_internal.cuh"

struct lsw_fno {
    int nz, nx, W, m, L;
    long long n;                 // nz * nx
    int M;                       // 2m modes per axis, M * M modes
    float2* params = nullptr;    // np entries
    float2* grads = nullptr;
    float2* adam_m = nullptr;
    float2* adam_v = nullptr;    // (second moments of re, im)
    long long np = 0;
    float2* Fz = nullptr;        // M x nz   rows of the DFT
    float2* FxT = nullptr;       // nx x M   (F_x)^T
    float2* Fxc = nullptr;       // M x nx   conj(F_x)
    // offsets into params
    long long oPT, op, oQT, oq;
    std::vector<long long> oR, oWT, ob;
};

namespace lsw {
namespace {

int gridn(long long n, int bs = 256) {
    long long g = (n + bs - 1) / bs;
    return (int)std::max<long long>(1, std::min<long long>(g, 152LL * 32));
}

__host__ __device__ inline float2 c1() { return make_float2(1.f, 0.f); }
__host__ __device__ inline float2 c0() { return make_float2(0.f, 0.f); }

__device__ __forceinline__ float gelu_f(float t) { return t * 0.5f * (1.f + erff(t * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_g(float t) {
    return 0.5f * (1.f + erff(t * 0.70710678118654752f)) + t * expf(-0.5f * t * t) * 0.3989422804014327f;
}

// rows of the DFT for the retained wavenumbers: F[a][i] = exp(-2 pi i k_a i / n)
__global__ void k_dft_rows(float2* F, int n, int m, int ld_rows_first) {
    const int M = 2 * m;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < M * n; e += gridDim.x * blockDim.x) {
        const int a = e % M, i = e / M;
        const int k = a < m ? a : n - 2 * m + a;
        double s, c;
        sincospi(-2.0 * (double)((long long)k * i % n) / n, &s, &c);
        const float2 v = make_float2((float)c, (float)s);
        // ld_rows_first: store M x n (element (a, i) at a + M i), else n x M transposed (i + n a)
        if (ld_rows_first) F[a + (long long)M * i] = v;
        else F[i + (long long)n * a] = v;
    }
}

__global__ void k_conj(const float2* a, float2* b, long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        b[e] = make_float2(a[e].x, -a[e].y);
}

// v[b][w][i] += bias[w]
__global__ void k_bias(float2* v, const float2* __restrict__ bias, long long n, int W, int B) {
    const long long tot = n * W * B;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const int w = (int)((e / n) % W);
        v[e].x += bias[w].x;
        v[e].y += bias[w].y;
    }
}

// z += bias; keep z; v = split-GELU(z) (or z)
__global__ void k_bias_act(float2* __restrict__ z, const float2* __restrict__ bias, float2* __restrict__ v, long long n,
                           int W, int B, int act) {
    const long long tot = n * W * B;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const int w = (int)((e / n) % W);
        float2 t = z[e];
        t.x += bias[w].x;
        t.y += bias[w].y;
        z[e] = t;
        v[e] = act ? make_float2(gelu_f(t.x), gelu_f(t.y)) : t;
    }
}

__global__ void k_act_grad(const float2* __restrict__ z, float2* __restrict__ g, long long tot) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const float2 t = z[e];
        float2 a = g[e];
        a.x *= gelu_g(t.x);
        a.y *= gelu_g(t.y);
        g[e] = a;
    }
}

// [b][w][mode] <-> [mode][b][w]: per mode a W x B column-major matrix
__global__ void k_bwm_to_mwb(const float2* __restrict__ s, float2* __restrict__ d, int B, int W, int MM) {
    const long long tot = (long long)B * W * MM;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const int md = (int)(e % MM);
        const long long r = e / MM;
        const int w = (int)(r % W), b = (int)(r / W);
        d[((long long)md * B + b) * W + w] = s[e];
    }
}
__global__ void k_mwb_to_bwm(const float2* __restrict__ s, float2* __restrict__ d, int B, int W, int MM) {
    const long long tot = (long long)B * W * MM;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const int md = (int)(e % MM);
        const long long r = e / MM;
        const int w = (int)(r % W), b = (int)(r / W);
        d[e] = s[((long long)md * B + b) * W + w];
    }
}

// G_y = 2 (y - t) / count; per-block partial sums of |y - t|^2
__global__ void k_loss(const float2* __restrict__ y, const float2* __restrict__ t, float2* __restrict__ g, long long tot,
                       float scale, double* part) {
    double s = 0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const float dx = y[e].x - t[e].x, dy = y[e].y - t[e].y;
        g[e] = make_float2(2.f * dx * scale, 2.f * dy * scale);
        s += (double)dx * dx + (double)dy * dy;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0;
        for (int i = 0; i < 8; ++i) a += red[i];
        part[blockIdx.x] = a;
    }
}

// out[w] = sum over b, i of g[b][w][i]   (one CTA per w)
__global__ void k_chan_sum(const float2* __restrict__ g, float2* __restrict__ out, long long n, int W, int B) {
    const int w = blockIdx.x;
    float sx = 0, sy = 0;
    for (int b = 0; b < B; ++b) {
        const float2* p = g + ((long long)b * W + w) * n;
        for (long long i = threadIdx.x; i < n; i += blockDim.x) {
            sx += p[i].x;
            sy += p[i].y;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
    }
    __shared__ float2 red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = make_float2(sx, sy);
    __syncthreads();
    if (threadIdx.x == 0) {
        float2 a = c0();
        for (int i = 0; i < 8; ++i) { a.x += red[i].x; a.y += red[i].y; }
        out[w] = a;
    }
}

// out = sum over b of part[b] (count elements each)
__global__ void k_batch_sum(const float2* __restrict__ part, float2* __restrict__ out, long long count, int B) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count; e += (long long)gridDim.x * blockDim.x) {
        float2 a = c0();
        for (int b = 0; b < B; ++b) { a.x += part[b * count + e].x; a.y += part[b * count + e].y; }
        out[e] = a;
    }
}

__global__ void k_adam(float2* __restrict__ w, const float2* __restrict__ g, float2* __restrict__ m, float2* __restrict__ v,
                       long long n, float lr, float b1, float b2, float eps, float c1_, float c2_) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float2 gg = g[e];
        float2 mm = m[e], vv = v[e];
        mm.x = b1 * mm.x + (1 - b1) * gg.x;
        mm.y = b1 * mm.y + (1 - b1) * gg.y;
        vv.x = b2 * vv.x + (1 - b2) * gg.x * gg.x;
        vv.y = b2 * vv.y + (1 - b2) * gg.y * gg.y;
        m[e] = mm;
        v[e] = vv;
        float2 ww = w[e];
        ww.x -= lr * (mm.x / c1_) / (sqrtf(vv.x / c2_) + eps);
        ww.y -= lr * (mm.y / c1_) / (sqrtf(vv.y / c2_) + eps);
        w[e] = ww;
    }
}

// Input channels of the preconditioner apply: x0 = v / s_b, x1 = chi / k0^2 + i k0 h
template <typename C>
__global__ void k_fno_input(const C* __restrict__ v, const double* __restrict__ inv_norm, const double* __restrict__ chi,
                            double ik02, float k0h, float2* __restrict__ x, long long n, int B) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n * B; e += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(e / n);
        const long long i = e - (long long)b * n;
        const double s = inv_norm[b];
        x[((long long)b * 2) * n + i] = make_float2((float)(v[e].x * s), (float)(v[e].y * s));
        x[((long long)b * 2 + 1) * n + i] = make_float2((float)(chi[i] * ik02), k0h);
    }
}

template <typename C>
__global__ void k_fno_output(const float2* __restrict__ y, const double* __restrict__ norm, C* __restrict__ z, long long n,
                             int B) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n * B; e += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(e / n);
        C o;
        o.x = y[e].x * norm[b];
        o.y = y[e].y * norm[b];
        z[e] = o;
    }
}

// t_b = e_b / ||r_b|| (complex128 or complex64 in, complex64 out)
template <typename C>
__global__ void k_scale_rows(const C* __restrict__ e, const double* __restrict__ inv_norm, float2* __restrict__ t,
                             long long n, int B) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n * B; q += (long long)gridDim.x * blockDim.x) {
        const double s = inv_norm[q / n];
        t[q] = make_float2((float)(e[q].x * s), (float)(e[q].y * s));
    }
}

// x_b channel 0 and t_b times exp(i phi_b)
__global__ void k_rotate_pairs(float2* __restrict__ x, float2* __restrict__ t, const float2* __restrict__ rot,
                               long long n, int B) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n * B; q += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(q / n);
        const long long i = q - (long long)b * n;
        const float2 w = rot[b];
        float2* xv = x + (long long)b * 2 * n + i;
        const float2 a = *xv, c = t[q];
        *xv = make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
        t[q] = make_float2(c.x * w.x - c.y * w.y, c.x * w.y + c.y * w.x);
    }
}

// per-block partial sums of |y - t|^2 and |t|^2 in FP64
__global__ void __launch_bounds__(256) k_err_sums(const float2* __restrict__ y, const float2* __restrict__ t,
                                                  long long tot, double* __restrict__ part) {
    __shared__ double sn[8], sd[8];
    double num = 0.0, den = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < tot; q += (long long)gridDim.x * blockDim.x) {
        const float2 a = y[q], c = t[q];
        const double dx = (double)a.x - c.x, dy = (double)a.y - c.y;
        num += dx * dx + dy * dy;
        den += (double)c.x * c.x + (double)c.y * c.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        num += __shfl_xor_sync(0xffffffffu, num, o);
        den += __shfl_xor_sync(0xffffffffu, den, o);
    }
    if ((threadIdx.x & 31) == 0) { sn[threadIdx.x >> 5] = num; sd[threadIdx.x >> 5] = den; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < 8; ++w) { a += sn[w]; b += sd[w]; }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
    }
}

__global__ void k_scale(float2* p, long long n, float a) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        p[e].x *= a;
        p[e].y *= a;
    }
}

__global__ void k_sqrt_inv(const double* __restrict__ n2, double* __restrict__ nrm, double* __restrict__ inv, int B) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const double s = sqrt(n2[b]);
    nrm[b] = s;
    inv[b] = s > 0 ? 1.0 / s : 0.0;
}

}  // namespace

// ------------------------------------------------------------- forward
// Activations kept for the backward pass.
struct FnoTape {
    int B = 0;
    std::vector<DevBuf*> bufs;
    float2 *x = nullptr, *y = nullptr;
    std::vector<float2*> v, z, Vh;     // v[0..L], z[0..L-1], Vh[0..L-1] ([b][w][mode])
    ~FnoTape() { for (auto* b : bufs) delete b; }
    float2* get(size_t elems, cudaStream_t st, lsw_status* s) {
        DevBuf* b = new (std::nothrow) DevBuf();
        if (!b) { *s = LSW_ERR_OOM; return nullptr; }
        bufs.push_back(b);
        const lsw_status r = b->alloc(sizeof(float2) * elems, st);
        if (r != LSW_OK) { *s = r; return nullptr; }
        return b->as<float2>();
    }
};

static lsw_status fno_forward(const lsw_fno* f, const float2* x, float2* y, int B, FnoTape& tp, cudaStream_t st) {
    const long long n = f->n;
    const int W = f->W, M = f->M, MM = M * M, nz = f->nz, nx = f->nx;
    const float2* P = f->params;
    lsw_status s = LSW_OK;
    tp.B = B;
    tp.v.assign(f->L + 1, nullptr);
    tp.z.assign(f->L, nullptr);
    tp.Vh.assign(f->L, nullptr);
    float2* T1 = tp.get((size_t)B * W * M * nx, st, &s);
    float2* Vt = tp.get((size_t)B * W * MM, st, &s);
    float2* Zt = tp.get((size_t)B * W * MM, st, &s);
    float2* Zh = tp.get((size_t)B * W * MM, st, &s);
    for (int l = 0; l <= f->L; ++l) tp.v[l] = tp.get((size_t)B * W * n, st, &s);
    for (int l = 0; l < f->L; ++l) {
        tp.z[l] = tp.get((size_t)B * W * n, st, &s);
        tp.Vh[l] = tp.get((size_t)B * W * MM, st, &s);
    }
    if (s != LSW_OK) return s;
    // lift: V0_b (n x W) = X_b (n x 2) P^T (2 x W) + p
    LSW_TRY(gemm<float>('N', 'N', (int)n, W, 2, c1(), x, (int)n, 2 * n, P + f->oPT, 2, 0, c0(), tp.v[0], (int)n, W * n, B, st));
    k_bias<<<gridn(n * W * B), 256, 0, st>>>(tp.v[0], P + f->op, n, W, B);
    LSW_LAUNCH_CHECK();
    for (int l = 0; l < f->L; ++l) {
        float2* v = tp.v[l];
        float2* z = tp.z[l];
        // Vh = Fz v FxT   (per sample and channel: M x M)
        LSW_TRY(gemm<float>('N', 'N', M, nx, nz, c1(), f->Fz, M, 0, v, nz, n, c0(), T1, M, (long long)M * nx, B * W, st));
        LSW_TRY(gemm<float>('N', 'N', M, M, nx, c1(), T1, M, (long long)M * nx, f->FxT, nx, 0, c0(), tp.Vh[l], M, MM,
                            B * W, st));
        // Zh[mode] = R[mode] Vh[mode]
        k_bwm_to_mwb<<<gridn((long long)B * W * MM), 256, 0, st>>>(tp.Vh[l], Vt, B, W, MM);
        LSW_LAUNCH_CHECK();
        LSW_TRY(gemm<float>('N', 'N', W, B, W, c1(), P + f->oR[l], W, (long long)W * W, Vt, W, (long long)W * B, c0(), Zt,
                            W, (long long)W * B, MM, st));
        k_mwb_to_bwm<<<gridn((long long)B * W * MM), 256, 0, st>>>(Zt, Zh, B, W, MM);
        LSW_LAUNCH_CHECK();
        // z = Fz^H (Zh conj(Fx)) / n
        LSW_TRY(gemm<float>('N', 'N', M, nx, M, c1(), Zh, M, MM, f->Fxc, M, 0, c0(), T1, M, (long long)M * nx, B * W, st));
        const float inv_n = 1.f / (float)n;
        LSW_TRY(gemm<float>('C', 'N', nz, nx, M, make_float2(inv_n, 0.f), f->Fz, M, 0, T1, M, (long long)M * nx, c0(), z,
                            nz, n, B * W, st));
        // z += V W^T; z += b; v' = sigma(z)
        LSW_TRY(gemm<float>('N', 'N', (int)n, W, W, c1(), v, (int)n, W * n, P + f->oWT[l], W, 0, c1(), z, (int)n, W * n, B,
                            st));
        k_bias_act<<<gridn(n * W * B), 256, 0, st>>>(z, P + f->ob[l], tp.v[l + 1], n, W, B, l < f->L - 1);
        LSW_LAUNCH_CHECK();
    }
    // project: y_b (n x 1) = x0_b + V_b Q^T + q  (the residual channel passes through)
    LSW_CUDA(cudaMemcpy2DAsync(y, sizeof(float2) * n, x, sizeof(float2) * 2 * n, sizeof(float2) * n, B,
                               cudaMemcpyDeviceToDevice, st));
    LSW_TRY(gemm<float>('N', 'N', (int)n, 1, W, c1(), tp.v[f->L], (int)n, W * n, P + f->oQT, W, 0, c1(), y, (int)n, n, B,
                        st));
    k_bias<<<gridn(n * B), 256, 0, st>>>(y, P + f->oq, n, 1, B);
    LSW_LAUNCH_CHECK();
    return LSW_OK;
}

static lsw_status fno_backward(lsw_fno* f, const float2* x, const float2* Gy, int B, FnoTape& tp, cudaStream_t st) {
    const long long n = f->n;
    const int W = f->W, M = f->M, MM = M * M, nz = f->nz, nx = f->nx;
    const float2* P = f->params;
    float2* G = f->grads;
    lsw_status s = LSW_OK;
    FnoTape wk;
    float2* Gv = wk.get((size_t)B * W * n, st, &s);
    float2* Gz = wk.get((size_t)B * W * n, st, &s);
    float2* T1 = wk.get((size_t)B * W * M * nx, st, &s);
    float2* GZh = wk.get((size_t)B * W * MM, st, &s);
    float2* GZt = wk.get((size_t)B * W * MM, st, &s);
    float2* Vt = wk.get((size_t)B * W * MM, st, &s);
    float2* GVt = wk.get((size_t)B * W * MM, st, &s);
    float2* GVh = wk.get((size_t)B * W * MM, st, &s);
    // per-sample partial weight gradients (W x W at most), summed over samples
    float2* part = wk.get((size_t)B * std::max<long long>((long long)W * W, 2LL * W), st, &s);
    if (s != LSW_OK) return s;
    // Q^T: sum_b V_b^H Gy_b;  q: sum Gy;  Gv = Gy Q^H... Gv_b (n x W) = Gy_b (n x 1) (Q^T)^H (1 x W)
    LSW_TRY(gemm<float>('C', 'N', W, 1, (int)n, c1(), tp.v[f->L], (int)n, W * n, Gy, (int)n, n, c0(), part, W, W, B, st));
    k_batch_sum<<<gridn(W), 256, 0, st>>>(part, G + f->oQT, W, B);
    LSW_LAUNCH_CHECK();
    k_chan_sum<<<1, 256, 0, st>>>(Gy, G + f->oq, n, 1, B);
    LSW_LAUNCH_CHECK();
    LSW_TRY(gemm<float>('N', 'C', (int)n, W, 1, c1(), Gy, (int)n, n, P + f->oQT, W, 0, c0(), Gv, (int)n, W * n, B, st));
    for (int l = f->L - 1; l >= 0; --l) {
        const long long tot = n * W * B;
        LSW_CUDA(cudaMemcpyAsync(Gz, Gv, sizeof(float2) * tot, cudaMemcpyDeviceToDevice, st));
        if (l < f->L - 1) {
            k_act_grad<<<gridn(tot), 256, 0, st>>>(tp.z[l], Gz, tot);
            LSW_LAUNCH_CHECK();
        }
        float2* v = tp.v[l];
        k_chan_sum<<<W, 256, 0, st>>>(Gz, G + f->ob[l], n, W, B);
        LSW_LAUNCH_CHECK();
        // W^T: sum_b V_b^H Gz_b
        LSW_TRY(gemm<float>('C', 'N', W, W, (int)n, c1(), v, (int)n, W * n, Gz, (int)n, W * n, c0(), part, W,
                            (long long)W * W, B, st));
        k_batch_sum<<<gridn((long long)W * W), 256, 0, st>>>(part, G + f->oWT[l], (long long)W * W, B);
        LSW_LAUNCH_CHECK();
        // G_Zh = Fz Gz FxT / n
        const float inv_n = 1.f / (float)n;
        LSW_TRY(gemm<float>('N', 'N', M, nx, nz, c1(), f->Fz, M, 0, Gz, nz, n, c0(), T1, M, (long long)M * nx, B * W, st));
        LSW_TRY(gemm<float>('N', 'N', M, M, nx, make_float2(inv_n, 0.f), T1, M, (long long)M * nx, f->FxT, nx, 0, c0(), GZh,
                            M, MM, B * W, st));
        k_bwm_to_mwb<<<gridn((long long)B * W * MM), 256, 0, st>>>(GZh, GZt, B, W, MM);
        LSW_LAUNCH_CHECK();
        k_bwm_to_mwb<<<gridn((long long)B * W * MM), 256, 0, st>>>(tp.Vh[l], Vt, B, W, MM);
        LSW_LAUNCH_CHECK();
        // G_R[mode] = GZt[mode] Vt[mode]^H ;  GVt[mode] = R[mode]^H GZt[mode]
        LSW_TRY(gemm<float>('N', 'C', W, W, B, c1(), GZt, W, (long long)W * B, Vt, W, (long long)W * B, c0(), G + f->oR[l],
                            W, (long long)W * W, MM, st));
        LSW_TRY(gemm<float>('C', 'N', W, B, W, c1(), P + f->oR[l], W, (long long)W * W, GZt, W, (long long)W * B, c0(), GVt,
                            W, (long long)W * B, MM, st));
        k_mwb_to_bwm<<<gridn((long long)B * W * MM), 256, 0, st>>>(GVt, GVh, B, W, MM);
        LSW_LAUNCH_CHECK();
        // Gv = Fz^H GVh conj(Fx)  +  Gz (W^T)^H
        LSW_TRY(gemm<float>('N', 'N', M, nx, M, c1(), GVh, M, MM, f->Fxc, M, 0, c0(), T1, M, (long long)M * nx, B * W, st));
        LSW_TRY(gemm<float>('C', 'N', nz, nx, M, c1(), f->Fz, M, 0, T1, M, (long long)M * nx, c0(), Gv, nz, n, B * W, st));
        LSW_TRY(gemm<float>('N', 'C', (int)n, W, W, c1(), Gz, (int)n, W * n, P + f->oWT[l], W, 0, c1(), Gv, (int)n, W * n, B,
                            st));
    }
    // lift: P^T: sum_b X_b^H Gv_b ; p: sum Gv
    k_chan_sum<<<W, 256, 0, st>>>(Gv, G + f->op, n, W, B);
    LSW_LAUNCH_CHECK();
    LSW_TRY(gemm<float>('C', 'N', 2, W, (int)n, c1(), x, (int)n, 2 * n, Gv, (int)n, W * n, c0(), part, 2, 2LL * W, B, st));
    k_batch_sum<<<gridn(2LL * W), 256, 0, st>>>(part, G + f->oPT, 2LL * W, B);
    LSW_LAUNCH_CHECK();
    return LSW_OK;
}

bool fno_matches(const lsw_fno* f, const lsw_green* g) { return g->nz == f->nz && g->nx == f->nx; }

lsw_status fno_apply_precond(const lsw_fno* f, const lsw_green* g, const double* chi, const void* v, void* z, int nb,
                             int prec, cudaStream_t st) {
    const long long n = f->n;
    if (!fno_matches(f, g)) return LSW_ERR_INVALID_ARG;
    DevBuf x, y, n2, nrm, inv;
    LSW_TRY(x.alloc(sizeof(float2) * 2 * n * nb, st));
    LSW_TRY(y.alloc(sizeof(float2) * n * nb, st));
    LSW_TRY(n2.alloc(sizeof(double) * nb, st));
    LSW_TRY(nrm.alloc(sizeof(double) * nb, st));
    LSW_TRY(inv.alloc(sizeof(double) * nb, st));
    if (prec == LSW_C128) LSW_TRY(norms2<double>((const double2*)v, n, nb, n2.as<double>(), st));
    else LSW_TRY(norms2<float>((const float2*)v, n, nb, n2.as<double>(), st));
    k_sqrt_inv<<<(nb + 255) / 256, 256, 0, st>>>(n2.as<double>(), nrm.as<double>(), inv.as<double>(), nb);
    LSW_LAUNCH_CHECK();
    const double ik02 = 1.0 / (g->k * g->k);
    const float k0h = (float)(g->k * g->h);
    if (prec == LSW_C128)
        k_fno_input<double2><<<gridn(n * nb), 256, 0, st>>>((const double2*)v, inv.as<double>(), chi, ik02, k0h,
                                                          x.as<float2>(), n, nb);
    else
        k_fno_input<float2><<<gridn(n * nb), 256, 0, st>>>((const float2*)v, inv.as<double>(), chi, ik02, k0h,
                                                         x.as<float2>(), n, nb);
    LSW_LAUNCH_CHECK();
    FnoTape tp;
    LSW_TRY(fno_forward(f, x.as<float2>(), y.as<float2>(), nb, tp, st));
    if (prec == LSW_C128)
        k_fno_output<double2><<<gridn(n * nb), 256, 0, st>>>(y.as<float2>(), nrm.as<double>(), (double2*)z, n, nb);
    else
        k_fno_output<float2><<<gridn(n * nb), 256, 0, st>>>(y.as<float2>(), nrm.as<double>(), (float2*)z, n, nb);
    LSW_LAUNCH_CHECK();
    return LSW_OK;
}

}  // namespace lsw

using namespace lsw;

extern "C" {

lsw_status lsw_fno_create(const lsw_fno_params* p, void* stream, lsw_fno** out) {
    if (!p || !out) return LSW_ERR_INVALID_ARG;
    *out = nullptr;
    if (p->nz < 2 || p->nx < 2 || p->width < 1 || p->width > 64 || p->modes < 1 || p->layers < 1 || p->layers > 16 ||
        2 * p->modes > p->nz || 2 * p->modes > p->nx)
        return LSW_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    lsw_fno* f = new (std::nothrow) lsw_fno();
    if (!f) return LSW_ERR_OOM;
    f->nz = p->nz; f->nx = p->nx; f->W = p->width; f->m = p->modes; f->L = p->layers;
    f->n = (long long)p->nz * p->nx;
    f->M = 2 * p->modes;
    const long long W = f->W, MM = (long long)f->M * f->M;
    long long o = 0;
    f->oPT = o; o += 2 * W;
    f->op = o; o += W;
    for (int l = 0; l < f->L; ++l) {
        f->oR.push_back(o); o += MM * W * W;
        f->oWT.push_back(o); o += W * W;
        f->ob.push_back(o); o += W;
    }
    f->oQT = o; o += W;
    f->oq = o; o += 1;
    f->np = o;
    lsw_status s = LSW_OK;
    auto al = [&](float2** ptr, long long cnt) {
        if (s == LSW_OK && cudaMalloc(ptr, sizeof(float2) * cnt) != cudaSuccess) s = LSW_ERR_OOM;
    };
    al(&f->params, f->np); al(&f->grads, f->np); al(&f->adam_m, f->np); al(&f->adam_v, f->np);
    al(&f->Fz, (long long)f->M * f->nz); al(&f->FxT, (long long)f->M * f->nx); al(&f->Fxc, (long long)f->M * f->nx);
    if (s != LSW_OK) { lsw_fno_destroy(f); return s; }
    cudaMemsetAsync(f->grads, 0, sizeof(float2) * f->np, st);
    cudaMemsetAsync(f->adam_m, 0, sizeof(float2) * f->np, st);
    cudaMemsetAsync(f->adam_v, 0, sizeof(float2) * f->np, st);
    k_dft_rows<<<gridn((long long)f->M * f->nz), 256, 0, st>>>(f->Fz, f->nz, f->m, 1);
    k_dft_rows<<<gridn((long long)f->M * f->nx), 256, 0, st>>>(f->FxT, f->nx, f->m, 0);
    {
        // Fxc = conj(F_x) as M x nx: conjugate-transpose of FxT via a temporary
        DevBuf tmp;
        s = tmp.alloc(sizeof(float2) * f->M * f->nx, st);
        if (s == LSW_OK) {
            k_dft_rows<<<gridn((long long)f->M * f->nx), 256, 0, st>>>(tmp.as<float2>(), f->nx, f->m, 1);
            k_conj<<<gridn((long long)f->M * f->nx), 256, 0, st>>>(tmp.as<float2>(), f->Fxc, (long long)f->M * f->nx);
        }
    }
    // Gaussian initial weights (Philox), scaled per tensor by 1/sqrt(fan-in); biases zero
    if (s == LSW_OK) {
        DevBuf w2, w3;
        s = w2.alloc(sizeof(uint32_t), st);
        if (s == LSW_OK) s = w3.alloc(sizeof(uint32_t), st);
        if (s == LSW_OK) {
            cudaMemsetAsync(w2.p, 0, 4, st);
            cudaMemsetAsync(w3.p, 0, 4, st);
            s = gaussian_fill<float>(f->params, (int)f->np, 1, f->np, 1, p->seed, w2.as<uint32_t>(), w3.as<uint32_t>(), st);
        }
        if (s == LSW_OK) {
            // fan-in scaling per tensor; biases start at zero
            auto scale = [&](long long off, long long cnt, float sc) {
                k_scale<<<gridn(cnt), 256, 0, st>>>(f->params + off, cnt, sc);
            };
            auto zero = [&](long long off, long long cnt) {
                cudaMemsetAsync(f->params + off, 0, sizeof(float2) * cnt, st);
            };
            scale(f->oPT, 2 * W, 1.f / std::sqrt(2.f));
            zero(f->op, W);
            for (int l = 0; l < f->L; ++l) {
                scale(f->oR[l], MM * W * W, 1.f / (float)W);
                scale(f->oWT[l], W * W, 1.f / std::sqrt((float)W));
                zero(f->ob[l], W);
            }
            scale(f->oQT, W, 1.f / std::sqrt((float)W));
            zero(f->oq, 1);
        }
    }
    if (s == LSW_OK && cudaGetLastError() != cudaSuccess) s = LSW_ERR_CUDA;
    if (s != LSW_OK) { lsw_fno_destroy(f); return s; }
    *out = f;
    return LSW_OK;
}

lsw_status lsw_fno_destroy(lsw_fno* f) {
    if (!f) return LSW_ERR_INVALID_ARG;
    for (float2* p : {f->params, f->grads, f->adam_m, f->adam_v, f->Fz, f->FxT, f->Fxc})
        if (p) cudaFree(p);
    delete f;
    return LSW_OK;
}

lsw_status lsw_fno_num_params(const lsw_fno* f, int64_t* count) {
    if (!f || !count) return LSW_ERR_INVALID_ARG;
    *count = f->np;
    return LSW_OK;
}

lsw_status lsw_fno_state(lsw_fno* f, int which, void* dst, const void* src, void* stream) {
    if (!f || (!dst && !src) || which < 0 || which > 3) return LSW_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    float2* buf = which == 0 ? f->params : which == 1 ? f->grads : which == 2 ? f->adam_m : f->adam_v;
    if (dst) LSW_CUDA(cudaMemcpyAsync(dst, buf, sizeof(float2) * f->np, cudaMemcpyDeviceToDevice, st));
    if (src) LSW_CUDA(cudaMemcpyAsync(buf, src, sizeof(float2) * f->np, cudaMemcpyDeviceToDevice, st));
    return LSW_OK;
}

lsw_status lsw_fno_forward(const lsw_fno* f, const void* x, void* y, int batch, void* stream) {
    if (!f || !x || !y || batch <= 0) return LSW_ERR_INVALID_ARG;
    FnoTape tp;
    return fno_forward(f, (const float2*)x, (float2*)y, batch, tp, reinterpret_cast<cudaStream_t>(stream));
}

lsw_status lsw_fno_loss_grad(lsw_fno* f, const void* x, const void* target, int batch, double* loss, void* grad,
                             void* stream) {
    if (!f || !x || !target || batch <= 0) return LSW_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const long long tot = f->n * batch;
    DevBuf y, gy, part;
    LSW_TRY(y.alloc(sizeof(float2) * tot, st));
    LSW_TRY(gy.alloc(sizeof(float2) * tot, st));
    const int nblk = 512;
    LSW_TRY(part.alloc(sizeof(double) * nblk, st));
    FnoTape tp;
    LSW_TRY(fno_forward(f, (const float2*)x, y.as<float2>(), batch, tp, st));
    k_loss<<<nblk, 256, 0, st>>>(y.as<float2>(), (const float2*)target, gy.as<float2>(), tot, 1.f / (float)tot,
                                 part.as<double>());
    LSW_LAUNCH_CHECK();
    LSW_TRY(fno_backward(f, (const float2*)x, gy.as<float2>(), batch, tp, st));
    if (grad) LSW_CUDA(cudaMemcpyAsync(grad, f->grads, sizeof(float2) * f->np, cudaMemcpyDeviceToDevice, st));
    if (loss) {
        std::vector<double> h(nblk);
        LSW_CUDA(cudaMemcpyAsync(h.data(), part.p, sizeof(double) * nblk, cudaMemcpyDeviceToHost, st));
        LSW_CUDA(cudaStreamSynchronize(st));
        double s = 0;
        for (double v : h) s += v;
        *loss = s / (double)tot;
    }
    return LSW_OK;
}

lsw_status lsw_fno_adam_step(lsw_fno* f, float lr, int32_t t, void* stream) {
    if (!f || !(lr > 0) || t < 1) return LSW_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const double b1 = 0.9, b2 = 0.999;
    const float c1_ = (float)(1.0 - std::pow(b1, (double)t)), c2_ = (float)(1.0 - std::pow(b2, (double)t));
    k_adam<<<gridn(f->np), 256, 0, st>>>(f->params, f->grads, f->adam_m, f->adam_v, f->np, lr, (float)b1, (float)b2,
                                         1e-8f, c1_, c2_);
    LSW_LAUNCH_CHECK();
    return LSW_OK;
}

lsw_status lsw_fno_pairs(const lsw_green* g, const double* chi, const void* r, const void* e, int nbatch, int prec,
                         void* x, void* t, void* stream) {
    if (!g || !chi || !r || !e || !x || !t || nbatch <= 0 || (prec != LSW_C128 && prec != LSW_C64))
        return LSW_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const long long n = (long long)g->nz * g->nx;
    DevBuf n2, nrm, inv;
    LSW_TRY(n2.alloc(sizeof(double) * nbatch, st));
    LSW_TRY(nrm.alloc(sizeof(double) * nbatch, st));
    LSW_TRY(inv.alloc(sizeof(double) * nbatch, st));
    if (prec == LSW_C128) LSW_TRY(norms2<double>((const double2*)r, n, nbatch, n2.as<double>(), st));
    else LSW_TRY(norms2<float>((const float2*)r, n, nbatch, n2.as<double>(), st));
    k_sqrt_inv<<<(nbatch + 255) / 256, 256, 0, st>>>(n2.as<double>(), nrm.as<double>(), inv.as<double>(), nbatch);
    LSW_LAUNCH_CHECK();
    const double ik02 = 1.0 / (g->k * g->k);
    const float k0h = (float)(g->k * g->h);
    if (prec == LSW_C128) {
        k_fno_input<double2><<<gridn(n * nbatch), 256, 0, st>>>((const double2*)r, inv.as<double>(), chi, ik02, k0h,
                                                               (float2*)x, n, nbatch);
        LSW_LAUNCH_CHECK();
        k_scale_rows<double2><<<gridn(n * nbatch), 256, 0, st>>>((const double2*)e, inv.as<double>(), (float2*)t, n,
                                                                nbatch);
    } else {
        k_fno_input<float2><<<gridn(n * nbatch), 256, 0, st>>>((const float2*)r, inv.as<double>(), chi, ik02, k0h,
                                                              (float2*)x, n, nbatch);
        LSW_LAUNCH_CHECK();
        k_scale_rows<float2><<<gridn(n * nbatch), 256, 0, st>>>((const float2*)e, inv.as<double>(), (float2*)t, n,
                                                               nbatch);
    }
    LSW_LAUNCH_CHECK();
    return LSW_OK;
}

lsw_status lsw_fno_rotate(void* x, void* t, int nbatch, int64_t n, const float* phases, void* stream) {
    if (!x || !t || !phases || nbatch <= 0 || n <= 0) return LSW_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    std::vector<float2> w(nbatch);
    for (int b = 0; b < nbatch; ++b) w[b] = make_float2((float)std::cos((double)phases[b]), (float)std::sin((double)phases[b]));
    DevBuf rot;
    LSW_TRY(rot.alloc(sizeof(float2) * nbatch, st));
    LSW_CUDA(cudaMemcpyAsync(rot.p, w.data(), sizeof(float2) * nbatch, cudaMemcpyHostToDevice, st));
    k_rotate_pairs<<<gridn((long long)n * nbatch), 256, 0, st>>>((float2*)x, (float2*)t, rot.as<float2>(), n, nbatch);
    LSW_LAUNCH_CHECK();
    // the host array w is read by the copy: wait before it goes out of scope
    LSW_CUDA(cudaStreamSynchronize(st));
    return LSW_OK;
}

lsw_status lsw_fno_error(const lsw_fno* f, const void* x, const void* t, int batch, double* num, double* den,
                         void* stream) {
    if (!f || !x || !t || !num || !den || batch <= 0) return LSW_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const long long tot = f->n * batch;
    DevBuf y, part;
    LSW_TRY(y.alloc(sizeof(float2) * tot, st));
    const int nblk = 256;
    LSW_TRY(part.alloc(sizeof(double) * 2 * nblk, st));
    FnoTape tp;
    LSW_TRY(fno_forward(f, (const float2*)x, y.as<float2>(), batch, tp, st));
    k_err_sums<<<nblk, 256, 0, st>>>(y.as<float2>(), (const float2*)t, tot, part.as<double>());
    LSW_LAUNCH_CHECK();
    std::vector<double> h(2 * nblk);
    LSW_CUDA(cudaMemcpyAsync(h.data(), part.p, sizeof(double) * 2 * nblk, cudaMemcpyDeviceToHost, st));
    LSW_CUDA(cudaStreamSynchronize(st));
    double a = 0.0, b = 0.0;
    for (int i = 0; i < nblk; ++i) { a += h[2 * i]; b += h[2 * i + 1]; }
    *num = a;
    *den = b;
    return LSW_OK;
}

lsw_status lsw_fno_apply(const lsw_fno* f, const lsw_green* g, const double* chi, const void* v, void* z, int nbatch,
                         int prec, void* stream) {
    if (!f || !g || !chi || !v || !z || nbatch <= 0 || (prec != LSW_C128 && prec != LSW_C64)) return LSW_ERR_INVALID_ARG;
    return fno_apply_precond(f, g, chi, v, z, nbatch, prec, reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
