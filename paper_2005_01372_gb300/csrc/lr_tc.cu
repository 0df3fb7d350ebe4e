// The H-matrix level products on the tcgen05 tensor cores, for factors kept
// as BF16 (re, im) pairs and complex64 vectors (the preconditioner apply of
// Sec. 2.4 on BF16 storage):
//     partial:  P_chunk = F_chunk^H X[rows of the sibling block]   (r x k)
//     apply:    Y[rows] += sum over levels of G_b[rows] T_b         (rows x k)
// with k <= 32 vectors.  Complex as real, as in the leaf products: an operand
// row holds (re, im) pairs along K, the other operand's real columns 0..31
// carry the real parts of the result and 32..63 the imaginary parts.  The
// vectors are split into BF16 hi + lo (two products), so the results carry
// the factors' BF16 rounding and hardly any of the vectors'.  FP32
// accumulation in tensor memory; bounded mbarrier waits (a timeout writes NaN).
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "lsw_internal.cuh"
#include "tc_ptx.cuh"

namespace lsw {
namespace {

using namespace tcx;

constexpr int LM = 128;                        // MMA rows (TMEM lanes)
constexpr int LN = 64;                         // real output columns
constexpr int LKC = 32;                        // complex K per stage
constexpr int LA = LM * 2 * LKC * 2;           // 16 KB: 128 rows x 64 BF16
constexpr int LB = LN * 2 * LKC * 2;           // 8 KB: 64 rows x 64 BF16
constexpr int LSTAGE = LA + 2 * LB;            // A, B hi, B lo
constexpr int LSMEM = 2 * LSTAGE + 64;
constexpr uint32_t LIDESC = idesc(1, LM, LN);
constexpr uint32_t LTMEM_COLS = 64;

__device__ int g_lr_tc_timeouts = 0;

// B'' rows for the vectors of one stage: thread (column jb = lane, complex K
// 8 gb .. 8 gb + 7 with gb = warp) writes its two kgroups of row jb (real
// part of the result) and of row 32 + jb (imaginary part).  conj = 1 builds
// the operand of F^H x: (xr, xi) and (xi, -xr); conj = 0 that of G t:
// (tr, -ti) and (ti, tr).
__device__ __forceinline__ void stage_b(unsigned char* Bhi, unsigned char* Blo, const float2 (&rb)[8], int jb, int gb,
                                        int conj) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t rh[4], rl[4], ih[4], il[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const float2 x = rb[4 * h + t];
            float xh, xl, yh, yl;
            split_bf16(x.x, xh, xl);
            split_bf16(x.y, yh, yl);
            if (conj) {
                rh[t] = pack_bf16(xh, yh);
                rl[t] = pack_bf16(xl, yl);
                ih[t] = pack_bf16(yh, -xh);
                il[t] = pack_bf16(yl, -xl);
            } else {
                rh[t] = pack_bf16(xh, -yh);
                rl[t] = pack_bf16(xl, -yl);
                ih[t] = pack_bf16(yh, xh);
                il[t] = pack_bf16(yl, xl);
            }
        }
        const int kg = 2 * gb + h;
        *reinterpret_cast<uint4*>(Bhi + kmaj(jb, kg)) = make_uint4(rh[0], rh[1], rh[2], rh[3]);
        *reinterpret_cast<uint4*>(Blo + kmaj(jb, kg)) = make_uint4(rl[0], rl[1], rl[2], rl[3]);
        *reinterpret_cast<uint4*>(Bhi + kmaj(jb + 32, kg)) = make_uint4(ih[0], ih[1], ih[2], ih[3]);
        *reinterpret_cast<uint4*>(Blo + kmaj(jb + 32, kg)) = make_uint4(il[0], il[1], il[2], il[3]);
    }
}

// Shared set-up of both kernels: two mbarriers, the abort flag and a TMEM
// accumulator of 64 columns.
struct TcCta {
    uint32_t mb[2];
    int* abort_flag;
    uint32_t tmem;
};

__device__ __forceinline__ TcCta tc_setup(unsigned char* sm) {
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + 2 * LSTAGE);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + 2 * LSTAGE + 16);
    TcCta c;
    c.abort_flag = reinterpret_cast<int*>(sm + 2 * LSTAGE + 32);
    c.mb[0] = smem_u32(&mbar[0]);
    c.mb[1] = smem_u32(&mbar[1]);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(c.mb[0]));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(c.mb[1]));
        asm volatile("fence.mbarrier_init.release.cluster;");
        *c.abort_flag = 0;
    }
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(LTMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    c.tmem = *tslot;
    return c;
}

// Issue the stage's MMAs (four K-steps of 16 BF16, B hi and lo) and commit
// them to the stage buffer's mbarrier.  Thread 0 only.
__device__ __forceinline__ void tc_issue(const TcCta& c, unsigned char* As, int buf, bool first) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    unsigned char* Bhi = As + LA;
    unsigned char* Blo = Bhi + LB;
    const uint32_t a = smem_u32(As), bh = smem_u32(Bhi), bl = smem_u32(Blo);
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
        const uint32_t o = ks * 256;   // 16 BF16 of K = two core matrices
        mma_bf16(c.tmem, sdesc(a + o), sdesc(bh + o), LIDESC, (!first || ks > 0) ? 1u : 0u);
        mma_bf16(c.tmem, sdesc(a + o), sdesc(bl + o), LIDESC, 1u);
    }
    mma_commit(c.mb[buf]);
}

// Wait for the last committed stage, then load the accumulator: thread's
// TMEM lane = its row.  Returns false when a wait gave up.
__device__ __forceinline__ bool tc_finish(const TcCta& c, int committed, float (&d)[LN]) {
    if (threadIdx.x == 0 && committed > 0) {
        const int s = committed - 1;
        if (!mbar_wait(c.mb[s & 1], (s >> 1) & 1)) *c.abort_flag = 1;
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const bool ok = *c.abort_flag == 0;
    const uint32_t taddr = c.tmem + ((uint32_t)((threadIdx.x >> 5) * 32) << 16);
#pragma unroll
    for (int col = 0; col < LN; col += 16) tmem_ld16(taddr + col, d + col);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    return ok;
}

__device__ __forceinline__ void tc_release(const TcCta& c) {
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(c.tmem), "r"(LTMEM_COLS));
}

// ------------------------------------------------------------- partials
// One CTA per chunk of CH rows of one level: A'' rows 0..r-1 are the columns
// of F over the chunk (each 32-row stage: 128 contiguous bytes per column),
// rows r..127 stay zero; B'' from the sibling block's rows of X.
__global__ void __launch_bounds__(128)
k_lr_partial_tc(LrLevels<float2, uint32_t> lv, int m, int r, int k, const float2* __restrict__ X, int swapA,
                float2* __restrict__ P) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int q = 0;
    while (q + 1 < lv.nlev && (int)blockIdx.x >= lv.chunk0[q + 1]) ++q;
    const int chn = blockIdx.x - lv.chunk0[q];
    const int CH = lv.ch[q], nb = lv.nb[q];
    const int row0 = chn * CH;
    const int j = row0 / nb, o = row0 - j * nb;
    const int src = swapA ? (j ^ 1) : j;
    const uint32_t* Fj = lv.F[q] + (long long)j * nb * r + o;
    const float2* Xg = X + (long long)src * nb + o;
    // A rows r..127 are zero in both buffers for the whole kernel
    for (int e = tid; e < 2 * (LA / 16); e += 128) {
        const int buf = e / (LA / 16), w = e - buf * (LA / 16);
        *reinterpret_cast<uint4*>(sm + buf * LSTAGE + 16 * w) = make_uint4(0u, 0u, 0u, 0u);
    }
    const TcCta c = tc_setup(sm);   // its barrier also orders the zeroing
    const int S = CH / LKC;
    uint4 ra[4];                               // r <= 64: 64 rows x 8 kgroups over 128 threads
    float2 rb[8];
    auto gload = [&](int s) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = tid + u * 128;
            const int i = e >> 3, kg = e & 7;
            ra[u] = (i < r) ? *reinterpret_cast<const uint4*>(Fj + (long long)i * nb + s * LKC + 4 * kg)
                            : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int t = 0; t < 8; ++t)
            rb[t] = lane < k ? Xg[(long long)lane * m + s * LKC + 8 * warp + t] : make_float2(0.f, 0.f);
    };
    gload(0);
    int committed = 0;
    for (int s = 0; s < S; ++s) {
        const int buf = s & 1;
        unsigned char* As = sm + buf * LSTAGE;
        if (tid == 0 && s >= 2 && !mbar_wait(c.mb[buf], ((s - 2) >> 1) & 1)) *c.abort_flag = 1;
        __syncthreads();
        if (*c.abort_flag) break;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = tid + u * 128;
            const int i = e >> 3, kg = e & 7;
            if (i < r) *reinterpret_cast<uint4*>(As + kmaj(i, kg)) = ra[u];
        }
        stage_b(As + LA, As + LA + LB, rb, lane, warp, 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (s + 1 < S) gload(s + 1);
        if (tid == 0) tc_issue(c, As, buf, s == 0);
        committed = s + 1;
    }
    float d[LN];
    const bool ok = tc_finish(c, committed, d) && committed == S;
    if (tid < r) {
        float2* out = P + (long long)blockIdx.x * r * k;
        for (int jj = 0; jj < k; ++jj)
            out[(long long)jj * r + tid] = ok ? make_float2(d[jj], d[32 + jj])
                                              : make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
    }
    if (!ok && tid == 0) atomicAdd(&g_lr_tc_timeouts, 1);
    tc_release(c);
}

// ---------------------------------------------------------------- apply
// One CTA per 128 rows of the node: for every level, the rows' factor G_b
// (thread = row, r entries with stride nb) times the block's T (r x k), in
// stages of 32 complex K; all levels accumulate in one TMEM tile, which is
// then added to Y.
__global__ void __launch_bounds__(128)
k_lr_apply_tc(LrLevels<float2, uint32_t> lv, int m, int r, int k, const float2* __restrict__ T, int swapC,
              float2* __restrict__ Y) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int i0 = blockIdx.x * LM;
    const long long nout = (long long)r * k;
    const TcCta c = tc_setup(sm);
    const int sq = (r + LKC - 1) / LKC;        // stages per level
    const int S = lv.nlev * sq;
    uint32_t ra[LKC];
    float2 rb[8];
    auto gload = [&](int g) {
        const int q = g / sq, s = g - q * sq;
        const int nb = lv.nb[q];
        const int b = i0 / nb, o = i0 - b * nb;
        const int bb = swapC ? (b ^ 1) : b;
        const uint32_t* Gb = lv.G[q] + (long long)bb * nb * r + o;
        const float2* Tb = T + (lv.t0[q] + bb) * nout;
        const int k0 = s * LKC;
#pragma unroll
        for (int kk = 0; kk < LKC; ++kk) ra[kk] = (k0 + kk < r) ? Gb[(long long)(k0 + kk) * nb + tid] : 0u;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int kt = k0 + 8 * warp + t;
            rb[t] = (lane < k && kt < r) ? Tb[(long long)lane * r + kt] : make_float2(0.f, 0.f);
        }
    };
    gload(0);
    int committed = 0;
    for (int g = 0; g < S; ++g) {
        const int buf = g & 1;
        unsigned char* As = sm + buf * LSTAGE;
        if (tid == 0 && g >= 2 && !mbar_wait(c.mb[buf], ((g - 2) >> 1) & 1)) *c.abort_flag = 1;
        __syncthreads();
        if (*c.abort_flag) break;
        // A'' row tid: kgroup q4 holds complex K 4 q4 .. 4 q4 + 3, (re, im) each
#pragma unroll
        for (int q4 = 0; q4 < 8; ++q4)
            *reinterpret_cast<uint4*>(As + kmaj(tid, q4)) =
                make_uint4(ra[4 * q4], ra[4 * q4 + 1], ra[4 * q4 + 2], ra[4 * q4 + 3]);
        stage_b(As + LA, As + LA + LB, rb, lane, warp, 0);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (g + 1 < S) gload(g + 1);
        if (tid == 0) tc_issue(c, As, buf, g == 0);
        committed = g + 1;
    }
    float d[LN];
    const bool ok = tc_finish(c, committed, d) && committed == S;
    const int row = i0 + tid;
    for (int jj = 0; jj < k && S > 0; ++jj) {
        float2* y = Y + (long long)jj * m + row;
        float2 v = *y;
        if (ok) {
            v.x += d[jj];
            v.y += d[32 + jj];
        } else {
            v = make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
        }
        *y = v;
    }
    if (!ok && tid == 0) atomicAdd(&g_lr_tc_timeouts, 1);
    tc_release(c);
}

}  // namespace

bool lr_tc_fits(const LrLevels<float2, uint32_t>& lv, int m, int r, int k) {
    if (!tc_gemm_enabled() || k < 1 || k > 32 || r < 1 || r > 64 || m % LM || lv.nlev < 1) return false;
    for (int q = 0; q < lv.nlev; ++q)
        if (lv.nb[q] % LM || lv.ch[q] % LKC) return false;
    return true;
}

lsw_status lr_partial_tc(const LrLevels<float2, uint32_t>& lv, int m, int r, int k, const float2* X, int swapA,
                         float2* P, cudaStream_t st) {
    static std::atomic<bool> attr{false};
    if (!attr.load()) {
        LSW_CUDA(cudaFuncSetAttribute(k_lr_partial_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, LSMEM));
        attr.store(true);
    }
    k_lr_partial_tc<<<lv.chunk0[lv.nlev], 128, LSMEM, st>>>(lv, m, r, k, X, swapA, P);
    LSW_LAUNCH_CHECK();
    return LSW_OK;
}

lsw_status lr_apply_tc(const LrLevels<float2, uint32_t>& lv, int m, int r, int k, const float2* T, int swapC,
                       float2* Y, cudaStream_t st) {
    static std::atomic<bool> attr{false};
    if (!attr.load()) {
        LSW_CUDA(cudaFuncSetAttribute(k_lr_apply_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, LSMEM));
        attr.store(true);
    }
    k_lr_apply_tc<<<m / LM, 128, LSMEM, st>>>(lv, m, r, k, T, swapC, Y);
    LSW_LAUNCH_CHECK();
    return LSW_OK;
}

}  // namespace lsw
