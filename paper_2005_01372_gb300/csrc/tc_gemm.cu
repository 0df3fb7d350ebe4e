// Batched complex FP32 GEMM on the 5th-generation tensor cores (tcgen05),
// for the products of the HODLR dense leaves with a block of vectors:
//     C_b = alpha A_b B_b,   A_b: M x K, B_b: K x N (N <= 32), column-major.
//
// Complex as real: with A'' (M x 2K) = [Re a_ik, Im a_ik] interleaved along
// K and B'' (2K x 64) whose columns 0..31 are [Re b_kj; -Im b_kj] and
// 32..63 are [Im b_kj; Re b_kj], the real product A'' B'' holds Re C in its
// first 32 columns and Im C in the last 32.
//
// FP32 accuracy from TF32 inputs ("3xTF32"): x = hi + lo with hi = x rounded
// to TF32 and lo = x - hi (exact in FP32); A B ~ Ahi Bhi + Ahi Blo + Alo Bhi,
// the dropped Alo Blo being ~2^-22 relative.  The accumulator stays in TMEM
// (FP32) for the whole K loop.
//
// One CTA of 128 threads owns 128 rows of one matrix.  Per stage of 16
// complex K (32 real): every thread loads its row of A and a slice of B into
// registers two stages ahead, splits them and stores hi/lo tiles into shared
// memory in the canonical K-major layout without swizzle (8-row x 16-byte core
// matrices, 128 B apart along K, 1024 B apart along rows); one thread issues
// 3 x 4 tcgen05.mma of 128 x 64 x 8 and commits them to the stage's mbarrier,
// which the producer waits on (bounded) before reusing that buffer.
#include <cuda_runtime.h>

#include <cuda_bf16.h>

#include <atomic>
#include <cstdint>

#include "lsw_internal.cuh"
#include "tc_ptx.cuh"

namespace lsw {
namespace {

constexpr int TC_M = 128;                       // rows per CTA (TMEM lanes)
constexpr int TC_KC = 16;                       // complex K per stage
constexpr int TC_NN = 64;                       // real output columns
constexpr int A_TILE = TC_M * 2 * TC_KC * 4;    // 16 KB: 128 rows x 32 TF32
constexpr int B_TILE = TC_NN * 2 * TC_KC * 4;   // 8 KB: 64 rows x 32 TF32
constexpr int STAGE = 2 * A_TILE + 2 * B_TILE;  // hi and lo of both
constexpr int TC_SMEM = 2 * STAGE + 64;         // two stages, barriers, TMEM slot
constexpr uint32_t TC_TMEM_COLS = 64;
// D F32 (bits 4-5 = 1), A and B TF32 (bits 7-9, 10-12 = 2), both K-major,
// N / 8 at bits 17-22, M / 16 at bits 24-28.
constexpr uint32_t TC_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_NN >> 3) << 17) |
                              ((uint32_t)(TC_M >> 4) << 24);
__device__ int g_tc_timeouts = 0;

using namespace tcx;

__global__ void __launch_bounds__(128)
k_cgemm_tc(const float2* __restrict__ A, int lda, long long sA, const float2* __restrict__ B, int ldb, long long sB,
           float2* __restrict__ Cm, int ldc, long long sC, int N, int K, float2 alpha) {
    extern __shared__ __align__(1024) unsigned char sm[];
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + 2 * STAGE);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + 2 * STAGE + 16);
    int* abort_flag = reinterpret_cast<int*>(sm + 2 * STAGE + 32);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int b = blockIdx.y, i0 = blockIdx.x * TC_M;
    const float2* Ab = A + b * sA + i0;
    const float2* Bb = B + b * sB;
    float2* Cb = Cm + b * sC + i0;
    const uint32_t mb0 = smem_u32(&mbar[0]), mb1 = smem_u32(&mbar[1]);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb0));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb1));
        asm volatile("fence.mbarrier_init.release.cluster;");
        *abort_flag = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tslot;

    const int S = K / TC_KC;
    const int jb = lane, gb = warp;              // B slice: column jb, complex k 4 gb .. 4 gb + 3
    // two register sets, each loaded two stages ahead of its use
    float2 ra0[TC_KC], rb0[4], ra1[TC_KC], rb1[4];
    auto gload = [&](int s, float2 (&ra)[TC_KC], float2 (&rb)[4]) {
        const int k0 = s * TC_KC;
#pragma unroll
        for (int kk = 0; kk < TC_KC; ++kk) ra[kk] = Ab[(long long)(k0 + kk) * lda + tid];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            rb[q] = jb < N ? Bb[(long long)jb * ldb + k0 + 4 * gb + q] : make_float2(0.f, 0.f);
    };
    int committed = 0;
    // one stage: wait for the buffer, split and store, refill the register
    // set for stage s + 2, issue the MMAs; false when a wait gave up
    auto stage = [&](int s, float2 (&ra)[TC_KC], float2 (&rb)[4]) -> bool {
        const int buf = s & 1;
        unsigned char* Ahi = sm + buf * STAGE;
        unsigned char* Alo = Ahi + A_TILE;
        unsigned char* Bhi = Alo + A_TILE;
        unsigned char* Blo = Bhi + B_TILE;
        if (tid == 0 && s >= 2 && !mbar_wait(buf ? mb1 : mb0, ((s - 2) >> 1) & 1)) *abort_flag = 1;
        __syncthreads();
        if (*abort_flag) return false;
        // A'' row tid: kgroup q holds [Re a(2q), Im a(2q), Re a(2q+1), Im a(2q+1)]
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            float h0, l0, h1, l1, h2, l2, h3, l3;
            split_tf32(ra[2 * q].x, h0, l0);
            split_tf32(ra[2 * q].y, h1, l1);
            split_tf32(ra[2 * q + 1].x, h2, l2);
            split_tf32(ra[2 * q + 1].y, h3, l3);
            *reinterpret_cast<float4*>(Ahi + kmaj(tid, q)) = make_float4(h0, h1, h2, h3);
            *reinterpret_cast<float4*>(Alo + kmaj(tid, q)) = make_float4(l0, l1, l2, l3);
        }
        // B'' rows jb (real part) and jb + 32 (imaginary part), kgroups 2 gb, 2 gb + 1
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float2 x0 = rb[2 * h], x1 = rb[2 * h + 1];
            float r0h, r0l, i0h, i0l, r1h, r1l, i1h, i1l;
            split_tf32(x0.x, r0h, r0l);
            split_tf32(x0.y, i0h, i0l);
            split_tf32(x1.x, r1h, r1l);
            split_tf32(x1.y, i1h, i1l);
            const int kg = 2 * gb + h;
            *reinterpret_cast<float4*>(Bhi + kmaj(jb, kg)) = make_float4(r0h, -i0h, r1h, -i1h);
            *reinterpret_cast<float4*>(Blo + kmaj(jb, kg)) = make_float4(r0l, -i0l, r1l, -i1l);
            *reinterpret_cast<float4*>(Bhi + kmaj(jb + 32, kg)) = make_float4(i0h, r0h, i1h, r1h);
            *reinterpret_cast<float4*>(Blo + kmaj(jb + 32, kg)) = make_float4(i0l, r0l, i1l, r1l);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (s + 2 < S) gload(s + 2, ra, rb);    // two stages of loads stay in flight
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(Bhi), bl = smem_u32(Blo);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                const uint32_t o = ks * 256;    // 8 real K = two core matrices
                mma_tf32(tmem, sdesc(ah + o), sdesc(bh + o), TC_IDESC, (s > 0 || ks > 0) ? 1u : 0u);
                mma_tf32(tmem, sdesc(ah + o), sdesc(bl + o), TC_IDESC, 1u);
                mma_tf32(tmem, sdesc(al + o), sdesc(bh + o), TC_IDESC, 1u);
            }
            mma_commit(buf ? mb1 : mb0);
        }
        committed = s + 1;
        return true;
    };
    gload(0, ra0, rb0);
    if (S > 1) gload(1, ra1, rb1);
    for (int s = 0; s < S; s += 2) {
        if (!stage(s, ra0, rb0)) break;
        if (s + 1 < S && !stage(s + 1, ra1, rb1)) break;
    }
    // the last commit covers every MMA issued before it
    if (tid == 0 && committed > 0) {
        const int s = committed - 1;
        if (!mbar_wait((s & 1) ? mb1 : mb0, (s >> 1) & 1)) *abort_flag = 1;
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const bool bad = *abort_flag != 0 || committed != S;
    // TMEM -> registers: warp w reads lanes 32 w .. 32 w + 31 (its rows)
    float d[TC_NN];
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
    for (int c = 0; c < TC_NN; c += 16) tmem_ld16(taddr + c, d + c);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const int row = warp * 32 + lane;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        if (j >= N) break;
        float2 o;
        if (bad) {
            o = make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
        } else {
            const float re = d[j], im = d[32 + j];
            o = make_float2(alpha.x * re - alpha.y * im, alpha.x * im + alpha.y * re);
        }
        Cb[(long long)j * ldc + row] = o;
    }
    if (bad && tid == 0) atomicAdd(&g_tc_timeouts, 1);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
}

// ---------------------------------------------------------------- BF16 A
// The same product with A stored as BF16 pairs (re, im) and B, C in FP32:
// kind::f16 MMAs (BF16 inputs, FP32 accumulation in TMEM).  B is split into
// BF16 hi + lo (two products), so the result carries A's BF16 rounding and
// hardly any of B's.  A stage is 32 complex K (64 BF16 = 128 B per row of
// A''): the tiles keep the byte layout of the TF32 kernel.
constexpr int TB_KC = 32;                          // complex K per stage
constexpr int TB_A = TC_M * 2 * TB_KC * 2;         // 16 KB
constexpr int TB_B = TC_NN * 2 * TB_KC * 2;        // 8 KB
constexpr int TB_STAGE = TB_A + 2 * TB_B;          // A, B hi, B lo
constexpr int TB_SMEM = 2 * TB_STAGE + 64;
// D F32 (bits 4-5 = 1), A and B BF16 (bits 7-9, 10-12 = 1), K-major, N / 8, M / 16
constexpr uint32_t TB_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_NN >> 3) << 17) |
                              ((uint32_t)(TC_M >> 4) << 24);

__global__ void __launch_bounds__(128)
k_cgemm_tc_bf16(const uint32_t* __restrict__ A, int lda, long long sA, const float2* __restrict__ B, int ldb,
                long long sB, float2* __restrict__ Cm, int ldc, long long sC, int N, int K, float2 alpha) {
    extern __shared__ __align__(1024) unsigned char sm[];
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + 2 * TB_STAGE);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + 2 * TB_STAGE + 16);
    int* abort_flag = reinterpret_cast<int*>(sm + 2 * TB_STAGE + 32);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int b = blockIdx.y, i0 = blockIdx.x * TC_M;
    const uint32_t* Ab = A + b * sA + i0;          // one BF16 pair per element
    const float2* Bb = B + b * sB;
    float2* Cb = Cm + b * sC + i0;
    const uint32_t mb0 = smem_u32(&mbar[0]), mb1 = smem_u32(&mbar[1]);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb0));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb1));
        asm volatile("fence.mbarrier_init.release.cluster;");
        *abort_flag = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tslot;
    const int S = K / TB_KC;
    const int jb = lane, gb = warp;                // B slice: column jb, complex k 8 gb .. 8 gb + 7
    uint32_t ra[TB_KC];
    float2 rb[8];
    auto gload = [&](int s) {
        const int k0 = s * TB_KC;
#pragma unroll
        for (int kk = 0; kk < TB_KC; ++kk) ra[kk] = Ab[(long long)(k0 + kk) * lda + tid];
#pragma unroll
        for (int q = 0; q < 8; ++q)
            rb[q] = jb < N ? Bb[(long long)jb * ldb + k0 + 8 * gb + q] : make_float2(0.f, 0.f);
    };
    gload(0);
    int committed = 0;
    for (int s = 0; s < S; ++s) {
        const int buf = s & 1;
        unsigned char* As = sm + buf * TB_STAGE;
        unsigned char* Bhi = As + TB_A;
        unsigned char* Blo = Bhi + TB_B;
        if (tid == 0 && s >= 2 && !mbar_wait(buf ? mb1 : mb0, ((s - 2) >> 1) & 1)) *abort_flag = 1;
        __syncthreads();
        if (*abort_flag) break;
        // A'' row tid: kgroup q (16 B) holds complex k = 4q .. 4q + 3, (re, im) each
#pragma unroll
        for (int q = 0; q < 8; ++q)
            *reinterpret_cast<uint4*>(As + kmaj(tid, q)) = make_uint4(ra[4 * q], ra[4 * q + 1], ra[4 * q + 2], ra[4 * q + 3]);
        // B'' rows jb ([Re b; -Im b]) and jb + 32 ([Im b; Re b]), kgroups 2 gb, 2 gb + 1
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint32_t rh[4], rl[4], ih[4], il[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const float2 x = rb[4 * h + t];
                float xh, xl, yh, yl;
                split_bf16(x.x, xh, xl);
                split_bf16(x.y, yh, yl);
                rh[t] = pack_bf16(xh, -yh);
                rl[t] = pack_bf16(xl, -yl);
                ih[t] = pack_bf16(yh, xh);
                il[t] = pack_bf16(yl, xl);
            }
            const int kg = 2 * gb + h;
            *reinterpret_cast<uint4*>(Bhi + kmaj(jb, kg)) = make_uint4(rh[0], rh[1], rh[2], rh[3]);
            *reinterpret_cast<uint4*>(Blo + kmaj(jb, kg)) = make_uint4(rl[0], rl[1], rl[2], rl[3]);
            *reinterpret_cast<uint4*>(Bhi + kmaj(jb + 32, kg)) = make_uint4(ih[0], ih[1], ih[2], ih[3]);
            *reinterpret_cast<uint4*>(Blo + kmaj(jb + 32, kg)) = make_uint4(il[0], il[1], il[2], il[3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (s + 1 < S) gload(s + 1);
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t a = smem_u32(As), bh = smem_u32(Bhi), bl = smem_u32(Blo);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                const uint32_t o = ks * 256;    // 16 BF16 of K = two core matrices
                mma_bf16(tmem, sdesc(a + o), sdesc(bh + o), TB_IDESC, (s > 0 || ks > 0) ? 1u : 0u);
                mma_bf16(tmem, sdesc(a + o), sdesc(bl + o), TB_IDESC, 1u);
            }
            mma_commit(buf ? mb1 : mb0);
        }
        committed = s + 1;
    }
    if (tid == 0 && committed > 0) {
        const int s = committed - 1;
        if (!mbar_wait((s & 1) ? mb1 : mb0, (s >> 1) & 1)) *abort_flag = 1;
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const bool bad = *abort_flag != 0 || committed != S;
    float d[TC_NN];
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll
    for (int c = 0; c < TC_NN; c += 16) tmem_ld16(taddr + c, d + c);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    const int row = warp * 32 + lane;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        if (j >= N) break;
        float2 o;
        if (bad) {
            o = make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
        } else {
            const float re = d[j], im = d[32 + j];
            o = make_float2(alpha.x * re - alpha.y * im, alpha.x * im + alpha.y * re);
        }
        Cb[(long long)j * ldc + row] = o;
    }
    if (bad && tid == 0) atomicAdd(&g_tc_timeouts, 1);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
}

std::atomic<int> g_tc_enabled{1};

}  // namespace

bool tc_gemm_enabled() { return g_tc_enabled.load() != 0; }
void tc_gemm_enable(bool on) { g_tc_enabled.store(on ? 1 : 0); }

bool tc_gemm_fits(int M, int N, int K) { return M > 0 && M % TC_M == 0 && K > 0 && K % TC_KC == 0 && N >= 1 && N <= 32; }

lsw_status cgemm_tc(const float2* A, int lda, long long sA, const float2* B, int ldb, long long sB, float2* C, int ldc,
                    long long sC, int M, int N, int K, float2 alpha, int batch, cudaStream_t st) {
    if (!tc_gemm_fits(M, N, K) || batch <= 0 || batch > 65535) return LSW_ERR_INVALID_ARG;
    static std::atomic<bool> attr{false};
    if (!attr.load()) {
        LSW_CUDA(cudaFuncSetAttribute(k_cgemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
        attr.store(true);
    }
    KTimer kt("leaf_tc", st, 8.0 * ((double)batch * M * K + (double)batch * K * N + (double)batch * M * N),
              8.0 * (double)batch * M * N * K);
    k_cgemm_tc<<<dim3(M / TC_M, batch), 128, TC_SMEM, st>>>(A, lda, sA, B, ldb, sB, C, ldc, sC, N, K, alpha);
    LSW_LAUNCH_CHECK();
    return LSW_OK;
}

bool tc_bf16_fits(int M, int N, int K) { return M > 0 && M % TC_M == 0 && K > 0 && K % TB_KC == 0 && N >= 1 && N <= 32; }

lsw_status cgemm_tc_bf16(const uint32_t* A, int lda, long long sA, const float2* B, int ldb, long long sB, float2* C,
                         int ldc, long long sC, int M, int N, int K, float2 alpha, int batch, cudaStream_t st) {
    if (!tc_bf16_fits(M, N, K) || batch <= 0 || batch > 65535) return LSW_ERR_INVALID_ARG;
    static std::atomic<bool> attr{false};
    if (!attr.load()) {
        LSW_CUDA(cudaFuncSetAttribute(k_cgemm_tc_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, TB_SMEM));
        attr.store(true);
    }
    KTimer kt("leaf_tc", st, 4.0 * (double)batch * M * K + 8.0 * ((double)batch * K * N + (double)batch * M * N),
              8.0 * (double)batch * M * N * K);
    k_cgemm_tc_bf16<<<dim3(M / TC_M, batch), 128, TB_SMEM, st>>>(A, lda, sA, B, ldb, sB, C, ldc, sC, N, K, alpha);
    LSW_LAUNCH_CHECK();
    return LSW_OK;
}

}  // namespace lsw

extern "C" lsw_status lsw_set_tensor_cores(int enable) {
    lsw::tc_gemm_enable(enable != 0);
    return LSW_OK;
}
