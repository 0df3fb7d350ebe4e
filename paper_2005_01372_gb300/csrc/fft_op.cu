// The Lippmann-Schwinger operator through zero-padded FFTs (Sec. 2.2, Eq. 4),
// and the Green table / spectra it multiplies by.
//
// A field on a (bz x bx) box is convolved with the Green table on the
// (2bz x 2bx) padded grid in three passes; the padded half of each axis is
// never stored:
//   pass A  (per column)  chi-multiply, zero-pad, FFT along z     -> T[kz][ix]
//   pass B  (per row kz)  zero-pad, FFT along x, multiply by the quarter
//                         spectrum, inverse FFT along x, crop      -> T[kz][ix]
//   pass C  (per column)  inverse FFT along z, crop, epilogue     -> y
// T holds 2bz x bx complex per field.  The spectrum carries the 1/(4 bz bx)
// of the inverse transform.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>

#include "fft.cuh"
#include "lsw_internal.cuh"

namespace lsw {

namespace {

template <typename R> struct FftCfg;
template <> struct FftCfg<float>  { static constexpr int NT = 256, MB4 = 8; };
template <> struct FftCfg<double> { static constexpr int NT = 256, MB4 = 4; };

// elements of one CTA's line set: nlines * P <= 4 * NT * MB4
template <typename R> constexpr int fft_capacity() { return 4 * FftCfg<R>::NT * FftCfg<R>::MB4; }

struct DevGeom {
    int bz, bx, logbz;
    const double* chi;
    int chi_ld;
    const int2* origin;
    int vpb;
};

__device__ __forceinline__ int2 box_origin(const DevGeom& g, int b) {
    return g.origin ? g.origin[b / g.vpb] : make_int2(0, 0);
}

// ----------------------------------------------------------------- pass A
template <typename R, int NT, int MB4>
__global__ void __launch_bounds__(NT)
k_pass_a(const typename Cx<R>::T* __restrict__ u, DevGeom geo, int pz, int logpz, int cx, int logcx,
         int lstride, const typename Cx<R>::T* __restrict__ tw, int twstep, int adjoint,
         typename Cx<R>::T* __restrict__ T) {
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    C* sm = reinterpret_cast<C*>(sm_raw);
    const int b = blockIdx.y;
    const int ix0 = blockIdx.x * cx;
    const int2 org = box_origin(geo, b);           // (z0, x0)
    const long long nbox = (long long)geo.bz * geo.bx;
    const C* ub = u + b * nbox;
    const int tot = cx * pz;
    for (int e = threadIdx.x; e < tot; e += NT) {
        const int c = e >> logpz, iz = e & (pz - 1);
        C v = czero<C>();
        if (iz < geo.bz) {
            const int ix = ix0 + c;
            v = ub[(long long)ix * geo.bz + iz];
            if (adjoint) {
                v.y = -v.y;
            } else {
                const R ch = (R)geo.chi[(long long)(org.y + ix) * geo.chi_ld + org.x + iz];
                v = cscale(v, ch);
            }
        }
        sm[c * lstride + iz] = v;
    }
    __syncthreads();
    smem_fft<C, NT, MB4>(sm, lstride, cx, pz, logpz, tw, twstep, false);
    C* Tb = T + (long long)b * pz * geo.bx;
    for (int e = threadIdx.x; e < tot; e += NT) {
        const int kz = e >> logcx, c = e & (cx - 1);
        Tb[(long long)kz * geo.bx + ix0 + c] = sm[c * lstride + kz];
    }
}

// ----------------------------------------------------------------- pass B
template <typename R, int NT, int MB4>
__global__ void __launch_bounds__(NT)
k_pass_b(typename Cx<R>::T* __restrict__ T, int bx, int pz, int px, int logpx, int rz, int logrz,
         int lstride, const typename Cx<R>::T* __restrict__ specq, int qz,
         const typename Cx<R>::T* __restrict__ tw, int twstep) {
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    C* sm = reinterpret_cast<C*>(sm_raw);
    const int b = blockIdx.y;
    const int kz0 = blockIdx.x * rz;
    C* Tb = T + (long long)b * pz * bx;
    const int tot = rz * px;
    for (int e = threadIdx.x; e < tot; e += NT) {
        const int r = e >> logpx, ix = e & (px - 1);
        sm[r * lstride + ix] = ix < bx ? Tb[(long long)(kz0 + r) * bx + ix] : czero<C>();
    }
    __syncthreads();
    smem_fft<C, NT, MB4>(sm, lstride, rz, px, logpx, tw, twstep, false);
    for (int e = threadIdx.x; e < tot; e += NT) {
        const int r = e >> logpx, kx = e & (px - 1);
        const int kz = kz0 + r;
        const int qx = min(kx, px - kx), qzz = min(kz, pz - kz);
        sm[r * lstride + kx] = cmul(sm[r * lstride + kx], specq[qx * qz + qzz]);
    }
    __syncthreads();
    smem_fft<C, NT, MB4>(sm, lstride, rz, px, logpx, tw, twstep, true);
    const int totc = rz * bx;
    for (int e = threadIdx.x; e < totc; e += NT) {
        const int r = e / bx, ix = e - r * bx;
        Tb[(long long)(kz0 + r) * bx + ix] = sm[r * lstride + ix];
    }
}

// ----------------------------------------------------------------- pass C
template <typename R, int NT, int MB4>
__global__ void __launch_bounds__(NT)
k_pass_c(const typename Cx<R>::T* __restrict__ T, DevGeom geo, int pz, int logpz, int cx, int logcx,
         int lstride, const typename Cx<R>::T* __restrict__ tw, int twstep, int mode,
         const typename Cx<R>::T* __restrict__ u, const typename Cx<R>::T* __restrict__ u0,
         typename Cx<R>::T* __restrict__ y) {
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    C* sm = reinterpret_cast<C*>(sm_raw);
    const int b = blockIdx.y;
    const int ix0 = blockIdx.x * cx;
    const C* Tb = T + (long long)b * pz * geo.bx;
    const int tot = cx * pz;
    for (int e = threadIdx.x; e < tot; e += NT) {
        const int kz = e >> logcx, c = e & (cx - 1);
        sm[c * lstride + kz] = Tb[(long long)kz * geo.bx + ix0 + c];
    }
    __syncthreads();
    smem_fft<C, NT, MB4>(sm, lstride, cx, pz, logpz, tw, twstep, true);
    const long long nbox = (long long)geo.bz * geo.bx;
    const int2 org = box_origin(geo, b);
    const int tote = cx * geo.bz;
    for (int e = threadIdx.x; e < tote; e += NT) {
        const int c = e >> geo.logbz, iz = e & (geo.bz - 1);
        const int ix = ix0 + c;
        const long long idx = b * nbox + (long long)ix * geo.bz + iz;
        C g = sm[c * lstride + iz];
        C out;
        switch (mode) {
            case LSW_OP_FORWARD:
                out = u0 ? cadd(u0[idx], g) : g;
                break;
            case LSW_OP_RESIDUAL:
                out = csub(u[idx], g);
                if (u0) out = csub(out, u0[idx]);
                break;
            case LSW_OP_ADJOINT: {
                const R ch = (R)geo.chi[(long long)(org.y + ix) * geo.chi_ld + org.x + iz];
                out = mk(g.x * ch, -g.y * ch);
                break;
            }
            default:
                out = g;
        }
        y[idx] = out;
    }
}

// ------------------------------------------------- register-FFT passes
// The same three passes with register-resident radix-8 line FFTs, for
// 8 <= 2bz, 2bx <= 2048.  Here T holds, per field, the 2bz x bx spectrum in
// kz-blocks: the kblk rows kz = kblk j .. kblk j + kblk - 1 (64 bytes of one
// column) lie next to each other for ix = 0, 1, ..., bx - 1, and the blocks
// follow each other.  A column's write (pass A) and read (pass C) then move
// whole 64-byte segments, and pass B reads and writes every kz-block as one
// contiguous run.
template <typename C> __host__ __device__ constexpr int kblk() { return 64 / (int)sizeof(C); }
template <typename C> __device__ __forceinline__ long long tile_index(int kz, int ix, int bx) {
    constexpr int KB = kblk<C>();
    return (long long)(kz / KB) * bx * KB + (long long)ix * KB + (kz % KB);
}
template <typename R, int LOGP>
__global__ void __launch_bounds__(256)
k_fa(const typename Cx<R>::T* __restrict__ u, DevGeom geo, const typename Cx<R>::T* __restrict__ tw,
     int twstep, int adjoint, typename Cx<R>::T* __restrict__ T) {
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    constexpr int pz = 1 << LOGP, Tz = pz >> 3, lpc = 256 / Tz;
    const int l = threadIdx.x / Tz, t = threadIdx.x - l * Tz;
    C* s = reinterpret_cast<C*>(sm_raw) + l * (pad8(pz) + 1);
    const int b = blockIdx.y;
    const int ix = blockIdx.x * lpc + l;
    const bool valid = ix < geo.bx;
    const int2 org = box_origin(geo, b);
    const C* ub = u + (long long)b * geo.bz * geo.bx + (long long)ix * geo.bz;
    C v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int iz = t + r * Tz;
        C x = czero<C>();
        if (valid && iz < geo.bz) {
            x = ub[iz];
            if (adjoint) {
                x.y = -x.y;
            } else {
                const R ch = (R)geo.chi[(long long)(org.y + ix) * geo.chi_ld + org.x + iz];
                x = cscale(x, ch);
            }
        }
        v[r] = x;
    }
    fft_line<C, LOGP>(v, s, t, tw, twstep, false);
    if (valid) {
        C* Tb = T + (long long)b * pz * geo.bx;
#pragma unroll
        for (int r = 0; r < 8; ++r) Tb[tile_index<C>(t + r * Tz, ix, geo.bx)] = v[r];
    }
}

// Pass B on kz-blocks.  A CTA owns nblk consecutive kz-blocks of one field
// (kblk rows each): it reads them as one contiguous run of memory, turns them
// into rows of a shared-memory tile (odd row stride), runs the x transforms
// of RC rows at a time (Tx threads per row, register radix-8 lines), and
// writes the run back.  Rows past the field's last kz-block are transformed
// as zeros and not stored, so every thread meets every barrier.
template <typename R, int LOGP, int NTB>
__global__ void __launch_bounds__(NTB)
k_fb(typename Cx<R>::T* __restrict__ T, int pz, int nblk, const typename Cx<R>::T* __restrict__ spt,
     const typename Cx<R>::T* __restrict__ tw, int twstep) {
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    constexpr int px = 1 << LOGP, bx = px >> 1, Tx = px >> 3, RC = NTB / Tx;
    constexpr int KB = kblk<C>();
    constexpr int TS = bx + 1;                                   // odd: transposing stores spread over banks
    C* tile = reinterpret_cast<C*>(sm_raw);                      // nblk * KB rows of TS
    const int l = threadIdx.x / Tx, t = threadIdx.x - l * Tx;
    C* s = tile + (size_t)nblk * KB * TS + (size_t)l * (pad8(px) + 1);
    const int b = blockIdx.y;
    const int kb0 = blockIdx.x * nblk;
    const int nb = min(nblk, pz / KB - kb0);                     // kz-blocks of this CTA
    const int nrows = nb * KB;
    C* run = T + (long long)b * pz * bx + (long long)kb0 * bx * KB;
    const int nrun = nrows * bx;
    for (int e = threadIdx.x; e < nrun; e += NTB) {
        const int blk = e / (bx * KB), w = e - blk * (bx * KB);
        const int ix = w / KB, r = w - ix * KB;
        tile[(blk * KB + r) * TS + ix] = run[e];
    }
    __syncthreads();
    const int rows_all = nblk * KB;
    for (int r0 = 0; r0 < rows_all; r0 += RC) {
        const int row = r0 + l;
        const bool live = row < nrows;
        const int kz = kb0 * KB + row;
        C v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int kx = t + q * Tx;
            v[q] = (live && kx < bx) ? tile[row * TS + kx] : czero<C>();
        }
        fft_line<C, LOGP>(v, s, t, tw, twstep, false);
        const int qzz = live ? min(kz, pz - kz) : 0;
        const C* sp = spt + (long long)qzz * (bx + 1);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int kx = t + q * Tx;
            v[q] = cmul(v[q], sp[min(kx, px - kx)]);
        }
        fft_line<C, LOGP>(v, s, t, tw, twstep, true);
        if (live) {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int kx = t + q * Tx;
                if (kx < bx) tile[row * TS + kx] = v[q];
            }
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nrun; e += NTB) {
        const int blk = e / (bx * KB), w = e - blk * (bx * KB);
        const int ix = w / KB, r = w - ix * KB;
        run[e] = tile[(blk * KB + r) * TS + ix];
    }
}

template <typename R, int LOGP>
__global__ void __launch_bounds__(256)
k_fc(const typename Cx<R>::T* __restrict__ T, DevGeom geo, const typename Cx<R>::T* __restrict__ tw,
     int twstep, int mode, const typename Cx<R>::T* __restrict__ u, const typename Cx<R>::T* __restrict__ u0,
     typename Cx<R>::T* __restrict__ y) {
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    constexpr int pz = 1 << LOGP, Tz = pz >> 3, lpc = 256 / Tz;
    const int l = threadIdx.x / Tz, t = threadIdx.x - l * Tz;
    C* s = reinterpret_cast<C*>(sm_raw) + l * (pad8(pz) + 1);
    const int b = blockIdx.y;
    const int ix = blockIdx.x * lpc + l;
    const bool valid = ix < geo.bx;
    const C* Tb = T + (long long)b * pz * geo.bx;
    C v[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = valid ? Tb[tile_index<C>(t + r * Tz, ix, geo.bx)] : czero<C>();
    fft_line<C, LOGP>(v, s, t, tw, twstep, true);
    if (!valid) return;
    const int2 org = box_origin(geo, b);
    const long long base = (long long)b * geo.bz * geo.bx + (long long)ix * geo.bz;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int iz = t + r * Tz;
        if (iz >= geo.bz) continue;
        const long long idx = base + iz;
        const C g = v[r];
        C out;
        switch (mode) {
            case LSW_OP_FORWARD:
                out = u0 ? cadd(u0[idx], g) : g;
                break;
            case LSW_OP_RESIDUAL:
                out = csub(u[idx], g);
                if (u0) out = csub(out, u0[idx]);
                break;
            case LSW_OP_ADJOINT: {
                const R ch = (R)geo.chi[(long long)(org.y + ix) * geo.chi_ld + org.x + iz];
                out = mk(g.x * ch, -g.y * ch);
                break;
            }
            default:
                out = g;
        }
        y[idx] = out;
    }
}

// ------------------------------------------------ generic strided 1D FFTs
// nlines lines of length P: element i of line l at data[l * lstep + i * estep].
template <int NT>
__global__ void __launch_bounds__(NT)
k_fft_strided64(double2* data, int P, int logP, int nlines, int lpc, long long lstep, long long estep,
                const double2* __restrict__ tw, int twstep, int inv) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    double2* sm = reinterpret_cast<double2*>(sm_raw);
    const int l0 = blockIdx.x * lpc;
    const int nl = min(lpc, nlines - l0);
    for (int e = threadIdx.x; e < nl * P; e += NT) {
        const int l = e >> logP, i = e & (P - 1);
        sm[l * P + i] = data[(l0 + l) * lstep + i * estep];
    }
    __syncthreads();
    smem_fft<double2, NT, 4>(sm, P, nl, P, logP, tw, twstep, inv != 0);
    for (int e = threadIdx.x; e < nl * P; e += NT) {
        const int l = e >> logP, i = e & (P - 1);
        data[(l0 + l) * lstep + i * estep] = sm[l * P + i];
    }
}

// ------------------------------------------------------------ Green table
// Cell-integrated Green's function (disk of equal area, radius a):
//   r > 0:  (i pi a / (2k)) J1(ka) H0(kr)
//   r = 0:  (i pi a / (2k)) H1(ka) - 1/k^2
__global__ void k_green_table(double2* table, int nz, int nx, double h, double k) {
    const int n = (nz + 1) * (nx + 1);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int dx = e / (nz + 1), dz = e - dx * (nz + 1);
        const double a = h * rsqrt(M_PI);
        const double ka = k * a;
        const double pre = M_PI * a / (2.0 * k);        // prefactor is i * pre
        double2 g;
        if (dx == 0 && dz == 0) {
            // i pre (J1 + i Y1) - 1/k^2
            g = make_double2(-pre * y1(ka) - 1.0 / (k * k), pre * j1(ka));
        } else {
            const double kr = k * h * sqrt((double)dz * dz + (double)dx * dx);
            const double s = pre * j1(ka);
            // i s (J0 + i Y0)
            g = make_double2(-s * y0(kr), s * j0(kr));
        }
        table[e] = g;
    }
}

// even extension of the table to (2bz x 2bx), column-major (2bx columns)
__global__ void k_extend(const double2* __restrict__ table, int nz, int bz, int bx, double2* ext) {
    const int pz = 2 * bz, px = 2 * bx;
    const long long n = (long long)pz * px;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(e / pz), iz = (int)(e - (long long)ix * pz);
        const int dx = min(ix, px - ix), dz = min(iz, pz - iz);
        ext[e] = table[dx * (nz + 1) + dz];
    }
}

__global__ void k_quarter(const double2* __restrict__ F, int bz, int bx, double2* q64, float2* q32, double2* t64,
                          float2* t32) {
    const int pz = 2 * bz;
    const int n = (bz + 1) * (bx + 1);
    const double sc = 1.0 / (4.0 * bz * bx);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int qx = e / (bz + 1), qz = e - qx * (bz + 1);
        const double2 v = F[(long long)qx * pz + qz];
        const double2 w = make_double2(v.x * sc, v.y * sc);
        const float2 f = make_float2((float)w.x, (float)w.y);
        q64[e] = w;
        q32[e] = f;
        t64[qz * (bx + 1) + qx] = w;
        t32[qz * (bx + 1) + qx] = f;
    }
}

__global__ void k_twiddles(double2* tw64, float2* tw32, int P) {
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < P; m += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(-2.0 * m / P, &s, &c);
        tw64[m] = make_double2(c, s);
        tw32[m] = make_float2((float)c, (float)s);
    }
}

__global__ void k_contrast(const double* __restrict__ vel, double* chi, long long n, double w2, double ic02) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const double c = vel[e];
        chi[e] = w2 * (1.0 / (c * c) - ic02);
    }
}

template <typename C>
__global__ void k_point_sources(const double2* __restrict__ table, int nz, int nx, const int2* __restrict__ pos,
                                int nsrc, double ih2, C* u0) {
    const long long n = (long long)nz * nx;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n * nsrc; e += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(e / n);
        const long long i = e - s * n;
        const int ix = (int)(i / nz), iz = (int)(i - (long long)ix * nz);
        const int dz = abs(iz - pos[s].x), dx = abs(ix - pos[s].y);
        const double2 g = table[dx * (nz + 1) + dz];
        C v;
        v.x = g.x * ih2;
        v.y = g.y * ih2;
        u0[e] = v;
    }
}

inline size_t pad8h(int i) { return (size_t)i + (size_t)(i >> 3); }

// Algorithmic bytes of one batched apply: per field read u (and u0) and
// write y; chi (FP64) and the quarter spectrum once per batch.
double op_bytes(size_t elem, int bz, int bx, int nb, bool has_u0, int) {
    const double cells = (double)bz * bx;
    return (double)elem * cells * (2.0 + (has_u0 ? 1.0 : 0.0)) * nb + 8.0 * cells + (double)elem * (bz + 1) * (bx + 1);
}
// 5 N log2 N per complex FFT: nx columns of 2nz, 2nz rows forward and back
// of 2nx, nx columns back; 6 per spectrum product.
double op_flops(int bz, int bx, int nb) {
    const double pz = 2.0 * bz, px = 2.0 * bx;
    const double fz = 5.0 * pz * std::log2(pz), fx = 5.0 * px * std::log2(px);
    return nb * (2.0 * bx * fz + 2.0 * pz * fx + 6.0 * pz * px);
}

int grid_for(long long n, int bs = 256) {
    long long g = (n + bs - 1) / bs;
    return (int)std::max<long long>(1, std::min<long long>(g, 152LL * 16));
}

}  // namespace

// Launch the register-FFT passes for a runtime log2 size (3..11).
template <typename K>
lsw_status set_smem(K k, std::atomic<bool>& done) {
    if (!done) {
        LSW_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
        done = true;
    }
    return LSW_OK;
}

#define LSW_LOG_SWITCH(lg, ...)                  \
    switch (lg) {                                \
        case 3: { constexpr int L_ = 3; __VA_ARGS__; break; }   \
        case 4: { constexpr int L_ = 4; __VA_ARGS__; break; }   \
        case 5: { constexpr int L_ = 5; __VA_ARGS__; break; }   \
        case 6: { constexpr int L_ = 6; __VA_ARGS__; break; }   \
        case 7: { constexpr int L_ = 7; __VA_ARGS__; break; }   \
        case 8: { constexpr int L_ = 8; __VA_ARGS__; break; }   \
        case 9: { constexpr int L_ = 9; __VA_ARGS__; break; }   \
        case 10: { constexpr int L_ = 10; __VA_ARGS__; break; } \
        case 11: { constexpr int L_ = 11; __VA_ARGS__; break; } \
        default: return LSW_ERR_UNSUPPORTED_SIZE;        \
    }

template <typename R>
lsw_status launch_fa(int lg, dim3 grid, size_t sm, cudaStream_t st, const typename Cx<R>::T* u, DevGeom dg,
                     const typename Cx<R>::T* tw, int tws, int adj, typename Cx<R>::T* work) {
    static std::atomic<bool> done[12];
    LSW_LOG_SWITCH(lg, {
        LSW_TRY(set_smem(k_fa<R, L_>, done[L_]));
        k_fa<R, L_><<<grid, 256, sm, st>>>(u, dg, tw, tws, adj, work);
        LSW_LAUNCH_CHECK();
    })
    return LSW_OK;
}

template <typename R, int NTB>
lsw_status launch_fb(int lg, dim3 grid, size_t sm, cudaStream_t st, typename Cx<R>::T* work, int pz, int nblk,
                     const typename Cx<R>::T* spt, const typename Cx<R>::T* tw, int tws) {
    static std::atomic<bool> done[12];
    LSW_LOG_SWITCH(lg, {
        if (L_ < 4 && NTB > 256) return LSW_ERR_UNSUPPORTED_SIZE;
        LSW_TRY(set_smem(k_fb<R, L_, NTB>, done[L_]));
        k_fb<R, L_, NTB><<<grid, NTB, sm, st>>>(work, pz, nblk, spt, tw, tws);
        LSW_LAUNCH_CHECK();
    })
    return LSW_OK;
}

template <typename R>
lsw_status launch_fc(int lg, dim3 grid, size_t sm, cudaStream_t st, const typename Cx<R>::T* work, DevGeom dg,
                     const typename Cx<R>::T* tw, int tws, int mode, const typename Cx<R>::T* u,
                     const typename Cx<R>::T* u0, typename Cx<R>::T* y) {
    static std::atomic<bool> done[12];
    LSW_LOG_SWITCH(lg, {
        LSW_TRY(set_smem(k_fc<R, L_>, done[L_]));
        k_fc<R, L_><<<grid, 256, sm, st>>>(work, dg, tw, tws, mode, u, u0, y);
        LSW_LAUNCH_CHECK();
    })
    return LSW_OK;
}

// ---------------------------------------------------------- pass tuning
// Variant of the operator passes per (2bz, 2bx, precision): 0 register FFT
// with 256-thread row CTAs in pass B, 1 the same with 512-thread row CTAs,
// 2 the shared-memory Stockham passes.  Chosen by lsw_autotune.
namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, int> g_tune;
thread_local int g_force_variant = -1;
}  // namespace

int op_variant(int pz, int px, int rsize) {
    if (g_force_variant >= 0) return g_force_variant;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(std::make_tuple(pz, px, rsize));
    return it == g_tune.end() ? 0 : it->second;
}

void op_force_variant(int v) { g_force_variant = v; }

void op_set_variant(int pz, int px, int rsize, int v) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[std::make_tuple(pz, px, rsize)] = v;
}

// ------------------------------------------------------------ op_apply
template <typename R>
lsw_status op_apply(const lsw_green* g, const Spectrum& sp, const OpGeom& geo, int mode,
                    const typename Cx<R>::T* u, const typename Cx<R>::T* u0, typename Cx<R>::T* y,
                    int nbatch, typename Cx<R>::T* work, cudaStream_t st) {
    typedef typename Cx<R>::T C;
    constexpr int NT = FftCfg<R>::NT, MB4 = FftCfg<R>::MB4, CAP = fft_capacity<R>();
    if (nbatch <= 0) return LSW_OK;
    const int bz = geo.bz, bx = geo.bx;
    const int pz = 2 * bz, px = 2 * bx;
    if (!is_pow2(bz) || !is_pow2(bx) || pz > CAP || px > CAP) return LSW_ERR_UNSUPPORTED_SIZE;
    if (sp.bz != bz || sp.bx != bx) return LSW_ERR_INVALID_ARG;
    const C* tw = reinterpret_cast<const C*>(sizeof(R) == 8 ? (const void*)g->tw64 : (const void*)g->tw32);
    const C* specq = reinterpret_cast<const C*>(sizeof(R) == 8 ? (const void*)sp.q64 : (const void*)sp.q32);

    DevGeom dg{bz, bx, ilog2(bz), geo.chi, geo.chi_ld, geo.origin, geo.vpb > 0 ? geo.vpb : 1};
    const int logpz = ilog2(pz), logpx = ilog2(px);
    const int variant = op_variant(pz, px, (int)sizeof(R));
    if (variant != 2 && pz >= 8 && px >= 8 && pz <= 2048 && px <= 2048 && sp.t32 && sp.t64) {
        const C* spt = reinterpret_cast<const C*>(sizeof(R) == 8 ? (const void*)sp.t64 : (const void*)sp.t32);
        const int ntb = (variant == 1 && px >= 16) ? 512 : 256;
        const int lz = 256 / (pz >> 3), lx = ntb / (px >> 3);
        const size_t smA = sizeof(C) * (size_t)lz * (pad8h(pz) + 1);
        // pass B: kz-blocks per CTA so that a CTA holds >= lx rows and about
        // 4096 entries, within the field's pz / kblk blocks
        constexpr int KB = kblk<C>();
        const int nkb = pz / KB;
        int nblk = std::max((lx + KB - 1) / KB, 4096 / (KB * bx));
        nblk = std::max(1, std::min(nblk, nkb));
        const size_t smB = sizeof(C) * ((size_t)nblk * KB * (bx + 1) + (size_t)lx * (pad8h(px) + 1));
        const int twz = g->twP / pz, twx = g->twP / px;
        dim3 gA((bx + lz - 1) / lz, nbatch), gB((nkb + nblk - 1) / nblk, nbatch);
        KTimer kt(sizeof(R) == 8 ? "operator_c128" : "operator_c64", st, op_bytes(sizeof(C), bz, bx, nbatch, u0 != nullptr, mode),
                  op_flops(bz, bx, nbatch));
        LSW_TRY(launch_fa<R>(logpz, gA, smA, st, u, dg, tw, twz, mode == LSW_OP_ADJOINT, work));
        if (ntb == 512) LSW_TRY((launch_fb<R, 512>(logpx, gB, smB, st, work, pz, nblk, spt, tw, twx)));
        else LSW_TRY((launch_fb<R, 256>(logpx, gB, smB, st, work, pz, nblk, spt, tw, twx)));
        LSW_TRY(launch_fc<R>(logpz, gA, smA, st, work, dg, tw, twz, mode, u, u0, y));
        return LSW_OK;
    }
    // columns per CTA for passes A and C, rows per CTA for pass B
    int cx = std::min(bx, std::max(1, CAP / pz));
    cx = std::min(cx, 16);
    int rz = std::min(pz, std::max(1, CAP / px));
    rz = std::min(rz, 16);
    const int lsa = pz + 1, lsb = px + 1;
    const size_t smA = (size_t)cx * lsa * sizeof(C), smB = (size_t)rz * lsb * sizeof(C);
    auto ka = k_pass_a<R, NT, MB4>;
    auto kb = k_pass_b<R, NT, MB4>;
    auto kc = k_pass_c<R, NT, MB4>;
    static std::atomic<bool> attr_done[2];
    if (!attr_done[sizeof(R) == 8]) {
        const int maxsm = 200 * 1024;
        LSW_CUDA(cudaFuncSetAttribute(ka, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
        LSW_CUDA(cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
        LSW_CUDA(cudaFuncSetAttribute(kc, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
        attr_done[sizeof(R) == 8] = true;
    }
    const int twz = g->twP / pz, twx = g->twP / px;
    dim3 gA(bx / cx, nbatch), gB(pz / rz, nbatch);
    ka<<<gA, NT, smA, st>>>(u, dg, pz, logpz, cx, ilog2(cx), lsa, tw, twz, mode == LSW_OP_ADJOINT, work);
    LSW_LAUNCH_CHECK();
    kb<<<gB, NT, smB, st>>>(work, bx, pz, px, logpx, rz, ilog2(rz), lsb, specq, bz + 1, tw, twx);
    LSW_LAUNCH_CHECK();
    kc<<<gA, NT, smA, st>>>(work, dg, pz, logpz, cx, ilog2(cx), lsa, tw, twz, mode, u, u0, y);
    LSW_LAUNCH_CHECK();
    return LSW_OK;
}

template lsw_status op_apply<float>(const lsw_green*, const Spectrum&, const OpGeom&, int, const float2*,
                                    const float2*, float2*, int, float2*, cudaStream_t);
template lsw_status op_apply<double>(const lsw_green*, const Spectrum&, const OpGeom&, int, const double2*,
                                     const double2*, double2*, int, double2*, cudaStream_t);

// ------------------------------------------------------- spectra and table
lsw_status build_spectrum(const lsw_green* g, int bz, int bx, Spectrum* out, cudaStream_t st) {
    if (bz > g->nz || bx > g->nx || !is_pow2(bz) || !is_pow2(bx)) return LSW_ERR_INVALID_ARG;
    const int pz = 2 * bz, px = 2 * bx;
    constexpr int NT = 256;
    const int cap = 4 * NT * 4;
    if (pz > cap || px > cap) return LSW_ERR_UNSUPPORTED_SIZE;
    DevBuf ext;
    LSW_TRY(ext.alloc(sizeof(double2) * (size_t)pz * px, st));
    double2* E = ext.as<double2>();
    k_extend<<<grid_for((long long)pz * px), 256, 0, st>>>(g->table, g->nz, bz, bx, E);
    LSW_LAUNCH_CHECK();
    auto kf = k_fft_strided64<NT>;
    LSW_CUDA(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    // along z: px lines of length pz, contiguous
    {
        const int lpc = std::max(1, std::min(px, cap / pz));
        kf<<<(px + lpc - 1) / lpc, NT, sizeof(double2) * lpc * pz, st>>>(E, pz, ilog2(pz), px, lpc, pz, 1,
                                                                         g->tw64, g->twP / pz, 0);
        LSW_LAUNCH_CHECK();
    }
    // along x: pz lines of length px, stride pz
    {
        const int lpc = std::max(1, std::min(pz, cap / px));
        kf<<<(pz + lpc - 1) / lpc, NT, sizeof(double2) * lpc * px, st>>>(E, px, ilog2(px), pz, lpc, 1, pz,
                                                                         g->tw64, g->twP / px, 0);
        LSW_LAUNCH_CHECK();
    }
    Spectrum s;
    s.bz = bz;
    s.bx = bx;
    const size_t nq = (size_t)(bz + 1) * (bx + 1);
    if (cudaMalloc(&s.q64, nq * sizeof(double2)) != cudaSuccess || cudaMalloc(&s.q32, nq * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&s.t64, nq * sizeof(double2)) != cudaSuccess || cudaMalloc(&s.t32, nq * sizeof(float2)) != cudaSuccess) {
        free_spectrum(&s);
        return LSW_ERR_OOM;
    }
    k_quarter<<<grid_for((long long)nq), 256, 0, st>>>(E, bz, bx, s.q64, s.q32, s.t64, s.t32);
    LSW_LAUNCH_CHECK();
    *out = s;
    return LSW_OK;
}

void free_spectrum(Spectrum* s) {
    if (s->q64) cudaFree(s->q64);
    if (s->q32) cudaFree(s->q32);
    if (s->t64) cudaFree(s->t64);
    if (s->t32) cudaFree(s->t32);
    s->q64 = nullptr;
    s->q32 = nullptr;
    s->t64 = nullptr;
    s->t32 = nullptr;
}

lsw_status green_init(lsw_green* g, cudaStream_t st) {
    const size_t nt = (size_t)(g->nz + 1) * (g->nx + 1);
    LSW_CUDA(cudaMalloc(&g->table, nt * sizeof(double2)));
    k_green_table<<<grid_for((long long)nt), 256, 0, st>>>(g->table, g->nz, g->nx, g->h, g->k);
    LSW_LAUNCH_CHECK();
    g->twP = 2 * std::max(g->nz, g->nx);
    LSW_CUDA(cudaMalloc(&g->tw64, g->twP * sizeof(double2)));
    LSW_CUDA(cudaMalloc(&g->tw32, g->twP * sizeof(float2)));
    k_twiddles<<<grid_for(g->twP), 256, 0, st>>>(g->tw64, g->tw32, g->twP);
    LSW_LAUNCH_CHECK();
    LSW_TRY(build_spectrum(g, g->nz, g->nx, &g->full, st));
    LSW_CUDA(cudaStreamSynchronize(st));
    return LSW_OK;
}

lsw_status contrast(const lsw_green* g, const double* vel, double* chi, cudaStream_t st) {
    const long long n = (long long)g->nz * g->nx;
    const double w = 2.0 * M_PI * g->freq;
    k_contrast<<<grid_for(n), 256, 0, st>>>(vel, chi, n, w * w, 1.0 / (g->c0 * g->c0));
    LSW_LAUNCH_CHECK();
    return LSW_OK;
}

lsw_status point_sources(const lsw_green* g, const int32_t* pos_host, int nsrc, int prec, void* u0,
                         cudaStream_t st) {
    for (int s = 0; s < nsrc; ++s) {
        if (pos_host[2 * s] < 0 || pos_host[2 * s] >= g->nz || pos_host[2 * s + 1] < 0 ||
            pos_host[2 * s + 1] >= g->nx)
            return LSW_ERR_INVALID_ARG;
    }
    DevBuf pos;
    LSW_TRY(pos.alloc(sizeof(int2) * nsrc, st));
    LSW_CUDA(cudaMemcpyAsync(pos.p, pos_host, sizeof(int2) * nsrc, cudaMemcpyHostToDevice, st));
    const long long n = (long long)g->nz * g->nx * nsrc;
    const double ih2 = 1.0 / (g->h * g->h);
    if (prec == LSW_C128)
        k_point_sources<double2><<<grid_for(n), 256, 0, st>>>(g->table, g->nz, g->nx, pos.as<int2>(), nsrc, ih2,
                                                              (double2*)u0);
    else
        k_point_sources<float2><<<grid_for(n), 256, 0, st>>>(g->table, g->nz, g->nx, pos.as<int2>(), nsrc, ih2,
                                                             (float2*)u0);
    LSW_LAUNCH_CHECK();
    // the host array is read by an async copy: wait before returning
    LSW_CUDA(cudaStreamSynchronize(st));
    return LSW_OK;
}

}  // namespace lsw
