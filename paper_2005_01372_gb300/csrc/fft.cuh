// Shared-memory Stockham FFT over a set of lines held by one CTA.
//
// Each stage of radix R (4, or 8 for the first stage of an odd power of two,
// or 2 for P = 2) maps butterfly j (0 <= j < P/R) with k = j mod Ns:
//     v_r = x[j + r P/R] * w^(r k P / (Ns R)),   r = 0..R-1
//     V   = DFT_R(v)
//     x'[(j / Ns) Ns R + k + r Ns] = V_r
// (the self-sorting "autosort" formulation: no bit reversal).  Every thread
// loads all of its butterflies into registers before a barrier and stores
// after it, so the stage is done in place.  The host guarantees
// nlines * P / 4 <= NT * MB4 (at most MB4 radix-4 butterflies per thread).
#pragma once

#include "lsw_internal.cuh"

namespace lsw {

template <typename C>
__device__ __forceinline__ C twiddle(const C* __restrict__ tw, int m, bool inv) {
    C w = tw[m];
    if (inv) w.y = -w.y;
    return w;
}

// multiply by -i (forward) or +i (inverse)
template <typename C>
__device__ __forceinline__ C rot90(C a, bool inv) { return inv ? mk(-a.y, a.x) : mk(a.y, -a.x); }

template <typename C>
__device__ __forceinline__ void dft4(C& v0, C& v1, C& v2, C& v3, bool inv) {
    C t0 = cadd(v0, v2), t1 = csub(v0, v2), t2 = cadd(v1, v3), t3 = rot90(csub(v1, v3), inv);
    v0 = cadd(t0, t2); v2 = csub(t0, t2); v1 = cadd(t1, t3); v3 = csub(t1, t3);
}

template <typename C>
__device__ __forceinline__ void dft8(C* v, bool inv) {
    // even / odd halves, then combine with w8^k
    C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4(e0, e1, e2, e3, inv);
    dft4(o0, o1, o2, o3, inv);
    typedef decltype(o0.x) R;
    const R s = (R)0.70710678118654752440;
    // w8^1 = (1 -+ i)/sqrt2, w8^2 = -+ i, w8^3 = (-1 -+ i)/sqrt2
    C w1o1 = inv ? mk((o1.x - o1.y) * s, (o1.x + o1.y) * s) : mk((o1.x + o1.y) * s, (o1.y - o1.x) * s);
    C w2o2 = rot90(o2, inv);
    C w3o3 = inv ? mk((-o3.x - o3.y) * s, (o3.x - o3.y) * s) : mk((o3.y - o3.x) * s, (-o3.x - o3.y) * s);
    v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
    v[1] = cadd(e1, w1o1); v[5] = csub(e1, w1o1);
    v[2] = cadd(e2, w2o2); v[6] = csub(e2, w2o2);
    v[3] = cadd(e3, w3o3); v[7] = csub(e3, w3o3);
}

// One radix-R stage over nlines lines of length P (line l at s + l*lstride).
template <typename C, int R, int NT, int MB>
__device__ __forceinline__ void fft_stage(C* s, int lstride, int nlines, int P, int logP, int Ns,
                                          const C* __restrict__ tw, int twstep, bool inv) {
    const int nbl = P / R;            // butterflies per line
    const int total = nlines * nbl;
    const int lognb = logP - (R == 8 ? 3 : (R == 4 ? 2 : 1));
    C v[MB][R];
#pragma unroll
    for (int i = 0; i < MB; ++i) {
        const int b = threadIdx.x + i * NT;
        if (b < total) {
            const int line = b >> lognb, j = b & (nbl - 1);
            const C* x = s + line * lstride;
            const int k = j & (Ns - 1);
#pragma unroll
            for (int r = 0; r < R; ++r) v[i][r] = x[j + r * nbl];
            if (Ns > 1) {
                const int m = k * (P / (Ns * R)) * twstep;
#pragma unroll
                for (int r = 1; r < R; ++r) v[i][r] = cmul(v[i][r], twiddle(tw, r * m, inv));
            }
            if (R == 4) dft4(v[i][0], v[i][1], v[i][2], v[i][3], inv);
            else if (R == 8) dft8(v[i], inv);
            else { C a = v[i][0]; v[i][0] = cadd(a, v[i][1]); v[i][1] = csub(a, v[i][1]); }
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < MB; ++i) {
        const int b = threadIdx.x + i * NT;
        if (b < total) {
            const int line = b >> lognb, j = b & (nbl - 1);
            C* x = s + line * lstride;
            const int k = j & (Ns - 1);
            const int base = (j - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; ++r) x[base + r * Ns] = v[i][r];
        }
    }
    __syncthreads();
}

// Full transform of nlines lines of length P = 2^logP (P >= 2).
// Caller synchronises before (data in smem) -- this routine ends synchronised.
template <typename C, int NT, int MB4>
__device__ void smem_fft(C* s, int lstride, int nlines, int P, int logP,
                         const C* __restrict__ tw, int twstep, bool inv) {
    if (P == 1) return;
    if (P == 2) { fft_stage<C, 2, NT, (MB4 * 2 > 16 ? 16 : MB4 * 2)>(s, lstride, nlines, P, logP, 1, tw, twstep, inv); return; }
    int Ns = 1;
    if (logP & 1) {
        fft_stage<C, 8, NT, (MB4 / 2 > 0 ? MB4 / 2 : 1)>(s, lstride, nlines, P, logP, Ns, tw, twstep, inv);
        Ns = 8;
    }
    while (Ns < P) {
        fft_stage<C, 4, NT, MB4>(s, lstride, nlines, P, logP, Ns, tw, twstep, inv);
        Ns *= 4;
    }
}

// ------------------------------------------------------------------------
// Register-resident line FFT.  A line of length P = 2^logP (8 <= P <= 2048)
// is held by T = P / 8 threads, thread t owning v[r] = x[t + r T].  One
// radix-2 or radix-4 stage (when log2 P is not a multiple of 3) is followed
// by radix-8 stages; between stages the line passes once through shared
// memory, indexed with one pad slot per 8 entries so that the strided
// Stockham stores spread over the banks.  The result comes back in the same
// layout, v[r] = X[t + r T]; the last stage needs no exchange.
__device__ __forceinline__ int pad8(int i) { return i + (i >> 3); }

template <typename C>
__device__ __forceinline__ void exch(C v[8], C* s, int t, int T) {
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = s[pad8(t + r * T)];
    __syncthreads();
}

template <typename C, int LOGP>
__device__ __forceinline__ void fft_line(C v[8], C* s, int t, const C* __restrict__ tw, int twstep, bool inv) {
    constexpr int P = 1 << LOGP;
    constexpr int T = P >> 3;
    constexpr int B = 1 << (LOGP % 3);
    int Ns = 1;
    if (B == 2) {
        // four radix-2 butterflies j = t + qT: inputs v[q], v[q + 4]; outputs y[2j], y[2j + 1]
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const C a = v[q], c = v[q + 4];
            const int j = t + q * T;
            s[pad8(2 * j)] = cadd(a, c);
            s[pad8(2 * j + 1)] = csub(a, c);
        }
        exch(v, s, t, T);
        Ns = 2;
    } else if (B == 4) {
        // two radix-4 butterflies j = t + qT: inputs v[q + 2r]; outputs y[4j + r]
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            C a0 = v[q], a1 = v[q + 2], a2 = v[q + 4], a3 = v[q + 6];
            dft4(a0, a1, a2, a3, inv);
            const int j = t + q * T;
            s[pad8(4 * j)] = a0;
            s[pad8(4 * j + 1)] = a1;
            s[pad8(4 * j + 2)] = a2;
            s[pad8(4 * j + 3)] = a3;
        }
        exch(v, s, t, T);
        Ns = 4;
    }
    constexpr int NST = LOGP / 3;          // radix-8 stages
#pragma unroll
    for (int st = 0; st < NST; ++st) {
        const int k = t & (Ns - 1);
        if (Ns > 1) {
            const int m = k * ((P >> 3) / Ns) * twstep;
#pragma unroll
            for (int r = 1; r < 8; ++r) v[r] = cmul(v[r], twiddle(tw, r * m, inv));
        }
        dft8(v, inv);
        if (st == NST - 1) break;
        const int base = (t - k) * 8 + k;
#pragma unroll
        for (int r = 0; r < 8; ++r) s[pad8(base + r * Ns)] = v[r];
        exch(v, s, t, T);
        Ns *= 8;
    }
}

}  // namespace lsw
