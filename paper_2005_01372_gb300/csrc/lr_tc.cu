// The H-matrix level products on the tcgen05 tensor cores, for factors kept
// as BF16 (re, im) pairs and complex64 vectors (the preconditioner apply of
// Sec. 2.4 on BF16 storage):
//     partial:  P_chunk = F_chunk^H X[rows of the sibling block]   (r x k)
//     apply:    Y[rows] += sum over levels of G_b[rows] T_b         (rows x k)
// with k <= 32 vectors.  Complex as real, as in the leaf products: an operand
// row holds (re, im) pairs along K, the other operand's real columns 0..NH-1
// carry the real parts of the result and NH..2NH-1 the imaginary parts (NH =
// 16 or 32, the vectors rounded up).  The vectors are split into BF16 hi + lo
// (two products), so the results carry the factors' BF16 rounding and hardly
// any of the vectors'.  FP32 accumulation in tensor memory.
//
// The factors are stored as their operand tiles (FAC_TILE_P, FAC_TILE_A), so
// a stage's A operand is one contiguous bulk copy (cp.async.bulk) into a ring
// of shared-memory buffers; the vectors are copied raw beside it and turned
// into the B operand by builder warps.  The CTAs are persistent and
// warp-specialised: each walks its share of the work items (chunks, row
// tiles) as one stream of stages, with a producer warp, an MMA warp, builder
// warps and epilogue warps synchronised by mbarriers, and two TMEM
// accumulators so that an item's epilogue overlaps the next item's stages.
// Every mbarrier wait is bounded; a wait that gives up makes the CTA write NaN
// to its items' outputs and count a timeout, after draining its copies in
// flight (bounded) and freeing its tensor memory.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "lsw_internal.cuh"
#include "tc_ptx.cuh"

namespace lsw {
namespace {

using namespace tcx;

constexpr int LM = 128;                        // MMA rows (TMEM lanes)
constexpr int LKC = 64;                        // rows (complex K) per partial stage
constexpr int XPAD = LKC * 8 + 16;             // smem stride of a raw column of a stage (+16 B: no bank conflicts)

__device__ int g_lr_tc_timeouts = 0;

__device__ __forceinline__ float qnan() { return __int_as_float(0x7fc00000); }

// The hi/lo BF16 words of four complex values x for the two B'' rows of one
// vector column: conj = 1 builds the operand of F^H x, rows (xr, xi) and
// (xi, -xr); conj = 0 that of G t, rows (tr, -ti) and (ti, tr).
__device__ __forceinline__ void b_words(const float2 (&x)[4], int conj, uint4& rh, uint4& rl, uint4& ih, uint4& il) {
    uint32_t a[4], b[4], c[4], d[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        float xh, xl, yh, yl;
        split_bf16(x[t].x, xh, xl);
        split_bf16(x[t].y, yh, yl);
        if (conj) {
            a[t] = pack_bf16(xh, yh);
            b[t] = pack_bf16(xl, yl);
            c[t] = pack_bf16(yh, -xh);
            d[t] = pack_bf16(yl, -xl);
        } else {
            a[t] = pack_bf16(xh, -yh);
            b[t] = pack_bf16(xl, -yl);
            c[t] = pack_bf16(yh, xh);
            d[t] = pack_bf16(yl, xl);
        }
    }
    rh = make_uint4(a[0], a[1], a[2], a[3]);
    rl = make_uint4(b[0], b[1], b[2], b[3]);
    ih = make_uint4(c[0], c[1], c[2], c[3]);
    il = make_uint4(d[0], d[1], d[2], d[3]);
}

// ------------------------------------------------ warp-specialised forms
// The same products with the roles of the stage chain on warps of their own,
// synchronised by mbarriers only (no block-wide barrier per stage):
//   warps 0..5  build B'' hi/lo of each stage from the raw vectors and arrive
//               on bready (one arrival per warp);
//   warp 6      producer: refills a ring slot once the MMAs that read it are
//               done (empty), with one bulk copy of the tiled factor and the
//               raw vector columns (full);
//   warp 7      one lane issues the MMAs of a stage once its B'' is ready and
//               commits them to empty (the slot), bfree (the B'' buffer) and,
//               at an item's last stage, accf (its accumulator);
//   warps 8..11 the epilogue: each reads its 32 TMEM lanes of a finished
//               accumulator and arrives on acce, which the MMA warp waits for
//               before it overwrites that accumulator two items later.
// Every wait is bounded; a role whose wait gives up sets the abort flag and
// leaves, the others then give up too (bounded), and the CTA writes NaN to
// all of its items' outputs after draining its copies.
constexpr int WS_THREADS = 384;
constexpr int WS_BUILDERS = 6;
constexpr int WS_PROD = 6, WS_MMA = 7, WS_EPI = 8;

struct WsBars {
    uint64_t* full;      // [ns]
    uint64_t* empty;     // [ns]
    uint64_t* bready;    // [2]
    uint64_t* bfree;     // [2]
    uint64_t* accf;      // [2]
    uint64_t* acce;      // [2]
    int* abort_flag;
    uint32_t* tslot;
    int* counts;         // [0] stages issued, [1] committed, [2] consumed by the builders
};
constexpr size_t ws_bar_bytes(int ns) { return 16 * (size_t)ns + 8 * 8 + 32; }

__device__ __forceinline__ WsBars ws_at(unsigned char* p, int ns) {
    WsBars b;
    b.full = reinterpret_cast<uint64_t*>(p);
    b.empty = b.full + ns;
    b.bready = b.empty + ns;
    b.bfree = b.bready + 2;
    b.accf = b.bfree + 2;
    b.acce = b.accf + 2;
    b.abort_flag = reinterpret_cast<int*>(b.acce + 2);
    b.tslot = reinterpret_cast<uint32_t*>(b.abort_flag + 1);
    b.counts = b.abort_flag + 2;
    return b;
}

__device__ __forceinline__ uint32_t ws_setup(const WsBars& b, int ns, uint32_t tcols) {
    if (threadIdx.x == 0) {
        for (int i = 0; i < ns; ++i) {
            mbar_init(smem_u32(b.full + i), 1);
            mbar_init(smem_u32(b.empty + i), 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(smem_u32(b.bready + i), WS_BUILDERS);
            mbar_init(smem_u32(b.bfree + i), 1);
            mbar_init(smem_u32(b.accf + i), 1);
            mbar_init(smem_u32(b.acce + i), 4);
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
        *b.abort_flag = 0;
        b.counts[0] = 0;
        b.counts[1] = 0;
        b.counts[2] = 0;
    }
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(b.tslot)),
                     "r"(tcols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    return *b.tslot;
}

// a plain arrival (no transaction bytes)
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ bool ws_wait(const WsBars& b, uint64_t* bar, uint32_t parity) {
    if (*reinterpret_cast<volatile int*>(b.abort_flag)) return false;
    if (mbar_wait(smem_u32(bar), parity)) return true;
    *b.abort_flag = 1;
    return false;
}

// End of a CTA: every role has left its loop.  Wait (bounded) for the copies
// issued and not consumed and for the last committed MMAs, free the tensor
// memory (warp 0 allocated it).  Returns whether the CTA aborted.
__device__ __forceinline__ bool ws_close(const WsBars& b, uint32_t tmem, uint32_t tcols, int ns) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const int issued = b.counts[0], committed = b.counts[1], consumed = b.counts[2];
        for (int s = consumed; s < issued; ++s)
            if (!mbar_wait(smem_u32(b.full + s % ns), (s / ns) & 1)) *b.abort_flag = 1;
        if (committed > 0) {
            const int s = committed - 1;
            if (!mbar_wait(smem_u32(b.empty + s % ns), (s / ns) & 1)) *b.abort_flag = 1;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    const bool aborted = *b.abort_flag != 0;
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols));
    return aborted;
}

// Partials: work item w = chunk w of the level list (chunk0 numbering): CH
// rows of one level, in stages of LKC = 64 rows.  A stage's A'' (rows = the
// rp factor columns, K = the 64 rows: eight K-step tiles) is one contiguous
// copy of rp x 256 bytes of the tiled F; the MMA's rows rp..127 read whatever
// follows in shared memory and land in accumulator rows that are never read.
// X's 64 rows of each of the k columns are copied raw (512 B each) and become
// B'' hi/lo in K-step tiles of 2 NH rows.
template <int NH>
__global__ void __launch_bounds__(WS_THREADS)
k_lr_partial_ws(LrLevels<float2, uint32_t> lv, int m, int r, int k, const float2* __restrict__ X, int swapA,
                float2* __restrict__ P, int ns) {
    constexpr int N = 2 * NH;
    constexpr uint32_t ID = idesc(1, LM, N);
    constexpr int KSP = LKC / 8;
    constexpr int KB = N * 32;
    constexpr int LBP = KSP * KB;
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwork = lv.chunk0[lv.nlev];
    const int rp = lv.rp;
    const uint32_t SA = (uint32_t)rp * 4 * LKC;
    const int SAS = (int)((SA + 1023) & ~1023u);
    const int XS = k * XPAD;
    unsigned char* Abuf = sm;
    unsigned char* Xbuf = sm + (size_t)ns * SAS;
    unsigned char* Bbuf = sm + (((size_t)ns * SAS + (size_t)ns * XS + 1023) & ~(size_t)1023);
    const WsBars bars = ws_at(Bbuf + 4 * LBP, ns);
    const uint32_t tmem = ws_setup(bars, ns, 2 * N);
    struct Item { int q, j, o, src, S; };
    auto item = [&](int w) {
        Item it;
        it.q = 0;
        while (it.q + 1 < lv.nlev && w >= lv.chunk0[it.q + 1]) ++it.q;
        const int CH = lv.ch[it.q], nb = lv.nb[it.q];
        const int row0 = (w - lv.chunk0[it.q]) * CH;
        it.j = row0 / nb;
        it.o = row0 - it.j * nb;
        it.src = swapA ? (it.j ^ 1) : it.j;
        it.S = CH / LKC;
        return it;
    };
    if (warp == WS_PROD) {
        int g = 0;
        bool go = true;
        for (int w = blockIdx.x; w < nwork && go; w += gridDim.x) {
            const Item it = item(w);
            const int nb = lv.nb[it.q];
            for (int s = 0; s < it.S; ++s, ++g) {
                const int slot = g % ns;
                if (g >= ns && !ws_wait(bars, bars.empty + slot, (uint32_t)((g / ns - 1) & 1))) { go = false; break; }
                const uint32_t fb = smem_u32(bars.full + slot);
                if (lane == 0) mbar_expect_tx(fb, SA + (uint32_t)k * LKC * 8u);
                __syncwarp();
                if (lane == 0)
                    bulk_g2s(smem_u32(Abuf + (size_t)slot * SAS),
                             lv.F[it.q] + fac_index(FAC_TILE_P, nb, r, rp, it.j, it.o + s * LKC, 0), SA, fb);
                if (lane < k)
                    bulk_g2s(smem_u32(Xbuf + (size_t)slot * XS + lane * XPAD),
                             X + (long long)it.src * nb + it.o + s * LKC + (long long)lane * m, (uint32_t)LKC * 8u, fb);
            }
        }
        if (lane == 0) bars.counts[0] = g;
    } else if (warp == WS_MMA) {
        if (lane == 0) {
            int g = 0, li = 0;
            bool go = true;
            for (int w = blockIdx.x; w < nwork && go; w += gridDim.x, ++li) {
                const Item it = item(w);
                if (li >= 2 && !ws_wait(bars, bars.acce + (li & 1), (uint32_t)(((li - 2) >> 1) & 1))) break;
                const uint32_t dt = tmem + (uint32_t)((li & 1) * N);
                for (int s = 0; s < it.S; ++s, ++g) {
                    const int slot = g % ns, bsel = g & 1;
                    if (!ws_wait(bars, bars.bready + bsel, (uint32_t)((g >> 1) & 1))) { go = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t a = smem_u32(Abuf + (size_t)slot * SAS);
                    const uint32_t bh = smem_u32(Bbuf + (size_t)bsel * 2 * LBP), bl = bh + LBP;
#pragma unroll
                    for (int ks = 0; ks < KSP; ++ks) {
                        const uint64_t da = sdesc_sbo(a + ks * rp * 32, 256);
                        mma_bf16(dt, da, sdesc_sbo(bh + ks * KB, 256), ID, (s > 0 || ks > 0) ? 1u : 0u);
                        mma_bf16(dt, da, sdesc_sbo(bl + ks * KB, 256), ID, 1u);
                    }
                    mma_commit(smem_u32(bars.empty + slot));
                    mma_commit(smem_u32(bars.bfree + bsel));
                    if (s == it.S - 1) mma_commit(smem_u32(bars.accf + (li & 1)));
                    bars.counts[1] = g + 1;
                }
            }
        }
        __syncwarp();
    } else if (warp >= WS_EPI) {
        const int row = (warp - WS_EPI) * 32 + lane;   // TMEM lane of this warp
        float d[N];
        int li = 0;
        for (int w = blockIdx.x; w < nwork; w += gridDim.x, ++li) {
            const bool ok = ws_wait(bars, bars.accf + (li & 1), (uint32_t)((li >> 1) & 1));
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t taddr = tmem + (uint32_t)((li & 1) * N) + ((uint32_t)((warp & 3) * 32) << 16);
#pragma unroll
            for (int col = 0; col < N; col += 16) tmem_ld16(taddr + col, d + col);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(bars.acce + (li & 1)));
            if (row < r) {
                float2* out = P + (long long)w * r * k;
#pragma unroll
                for (int jj = 0; jj < NH; ++jj)
                    if (jj < k) out[(long long)jj * r + row] = make_float2(d[jj], d[NH + jj]);
            }
        }
    } else {
        // builders: warp (0..5) takes K-steps warp, warp + 6 of each stage
        int g = 0;
        bool go = true;
        for (int w = blockIdx.x; w < nwork && go; w += gridDim.x) {
            const Item it = item(w);
            for (int s = 0; s < it.S; ++s, ++g) {
                const int slot = g % ns, bsel = g & 1;
                if (!ws_wait(bars, bars.full + slot, (uint32_t)((g / ns) & 1))) { go = false; break; }
                if (g >= 2 && !ws_wait(bars, bars.bfree + bsel, (uint32_t)(((g - 2) >> 1) & 1))) { go = false; break; }
                unsigned char* Bhi = Bbuf + (size_t)bsel * 2 * LBP;
                unsigned char* Blo = Bhi + LBP;
                if (lane < NH) {
                    const float4* xs = reinterpret_cast<const float4*>(Xbuf + (size_t)slot * XS + lane * XPAD);
                    for (int ks = warp; ks < KSP; ks += WS_BUILDERS) {
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            float2 x[4];
#pragma unroll
                            for (int t = 0; t < 2; ++t) {
                                const float4 v = lane < k ? xs[4 * ks + 2 * h + t] : make_float4(0.f, 0.f, 0.f, 0.f);
                                x[2 * t] = make_float2(v.x, v.y);
                                x[2 * t + 1] = make_float2(v.z, v.w);
                            }
                            uint4 rh, rl, ih, il;
                            b_words(x, 1, rh, rl, ih, il);
                            const int ob = ks * KB;
                            *reinterpret_cast<uint4*>(Bhi + ob + kstep_off(lane, h)) = rh;
                            *reinterpret_cast<uint4*>(Blo + ob + kstep_off(lane, h)) = rl;
                            *reinterpret_cast<uint4*>(Bhi + ob + kstep_off(lane + NH, h)) = ih;
                            *reinterpret_cast<uint4*>(Blo + ob + kstep_off(lane + NH, h)) = il;
                        }
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(bars.bready + bsel));
            }
        }
        if (warp == 0 && lane == 0) bars.counts[2] = g;
    }
    if (ws_close(bars, tmem, 2 * N, ns)) {
        for (int w = blockIdx.x; w < nwork; w += gridDim.x)
            for (int e = tid; e < r * k; e += blockDim.x)
                P[(long long)w * r * k + e] = make_float2(qnan(), qnan());
        if (tid == 0) atomicAdd(&g_lr_tc_timeouts, 1);
    }
}

// Apply: work item = 128 rows of the node, one stage per level.  The tiled G
// holds the 128 rows' rp columns as rp / 8 contiguous 4 KB K-step tiles: one
// copy.  The block's T (r x k, column-major) comes raw, a column at a time,
// and becomes B'' hi/lo (rp / 8 K-step tiles of 2 NH rows).  All levels
// accumulate in one TMEM accumulator, which the epilogue adds to Y.
template <int NH>
__global__ void __launch_bounds__(WS_THREADS)
k_lr_apply_ws(LrLevels<float2, uint32_t> lv, int m, int r, int k, const float2* __restrict__ T, int swapC,
              float2* __restrict__ Y, int ns) {
    constexpr int N = 2 * NH;
    constexpr uint32_t ID = idesc(1, LM, N);
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwork = m / LM;
    const long long nout = (long long)r * k;
    const int rp = lv.rp, nks = rp >> 3;
    const uint32_t SA = (uint32_t)nks * 4096u;
    const int TP = r * 8 + 16;
    const int TS = (k * TP + 127) & ~127;
    const int KB = N * 32;
    const int BB = nks * KB;
    unsigned char* Abuf = sm;
    unsigned char* Tbuf = sm + (size_t)ns * SA;
    unsigned char* Bbuf = sm + (((size_t)ns * SA + (size_t)ns * TS + 1023) & ~(size_t)1023);
    const WsBars bars = ws_at(Bbuf + 4 * BB, ns);
    const uint32_t tmem = ws_setup(bars, ns, 2 * N);
    const int S = lv.nlev;
    if (warp == WS_PROD) {
        int g = 0;
        bool go = true;
        for (int w = blockIdx.x; w < nwork && go; w += gridDim.x) {
            const int i0 = w * LM;
            for (int s = 0; s < S; ++s, ++g) {
                const int slot = g % ns;
                if (g >= ns && !ws_wait(bars, bars.empty + slot, (uint32_t)((g / ns - 1) & 1))) { go = false; break; }
                const int nb = lv.nb[s];
                const int b = i0 / nb, o = i0 - b * nb;
                const int bb = swapC ? (b ^ 1) : b;
                const uint32_t fb = smem_u32(bars.full + slot);
                if (lane == 0) mbar_expect_tx(fb, SA + (uint32_t)k * r * 8u);
                __syncwarp();
                if (lane == 0)
                    bulk_g2s(smem_u32(Abuf + (size_t)slot * SA), lv.G[s] + fac_index(FAC_TILE_A, nb, r, rp, bb, o, 0),
                             SA, fb);
                if (lane < k)
                    bulk_g2s(smem_u32(Tbuf + (size_t)slot * TS + lane * TP),
                             T + (lv.t0[s] + bb) * nout + (long long)lane * r, (uint32_t)r * 8u, fb);
            }
        }
        if (lane == 0) bars.counts[0] = g;
    } else if (warp == WS_MMA) {
        if (lane == 0) {
            int g = 0, li = 0;
            bool go = true;
            for (int w = blockIdx.x; w < nwork && go; w += gridDim.x, ++li) {
                if (li >= 2 && !ws_wait(bars, bars.acce + (li & 1), (uint32_t)(((li - 2) >> 1) & 1))) break;
                const uint32_t dt = tmem + (uint32_t)((li & 1) * N);
                for (int s = 0; s < S; ++s, ++g) {
                    const int slot = g % ns, bsel = g & 1;
                    if (!ws_wait(bars, bars.bready + bsel, (uint32_t)((g >> 1) & 1))) { go = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t a = smem_u32(Abuf + (size_t)slot * SA);
                    const uint32_t bh = smem_u32(Bbuf + (size_t)bsel * 2 * BB), bl = bh + BB;
                    for (int ks = 0; ks < nks; ++ks) {
                        const uint64_t da = sdesc_sbo(a + ks * 4096, 256);
                        mma_bf16(dt, da, sdesc_sbo(bh + ks * KB, 256), ID, (s > 0 || ks > 0) ? 1u : 0u);
                        mma_bf16(dt, da, sdesc_sbo(bl + ks * KB, 256), ID, 1u);
                    }
                    mma_commit(smem_u32(bars.empty + slot));
                    mma_commit(smem_u32(bars.bfree + bsel));
                    if (s == S - 1) mma_commit(smem_u32(bars.accf + (li & 1)));
                    bars.counts[1] = g + 1;
                }
            }
        }
        __syncwarp();
    } else if (warp >= WS_EPI) {
        float d[N];
        int li = 0;
        for (int w = blockIdx.x; w < nwork; w += gridDim.x, ++li) {
            if (!ws_wait(bars, bars.accf + (li & 1), (uint32_t)((li >> 1) & 1))) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t taddr = tmem + (uint32_t)((li & 1) * N) + ((uint32_t)((warp & 3) * 32) << 16);
#pragma unroll
            for (int col = 0; col < N; col += 16) tmem_ld16(taddr + col, d + col);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(bars.acce + (li & 1)));
            const int row = w * LM + (warp & 3) * 32 + lane;
#pragma unroll
            for (int jj = 0; jj < NH; ++jj) {
                if (jj >= k) continue;
                float2* y = Y + (long long)jj * m + row;
                const float2 v = *y;
                *y = make_float2(v.x + d[jj], v.y + d[NH + jj]);
            }
        }
    } else {
        // builders: warp (0..5) takes K-steps warp, warp + 6 of each level
        int g = 0;
        bool go = true;
        for (int w = blockIdx.x; w < nwork && go; w += gridDim.x) {
            for (int s = 0; s < S; ++s, ++g) {
                const int slot = g % ns, bsel = g & 1;
                if (!ws_wait(bars, bars.full + slot, (uint32_t)((g / ns) & 1))) { go = false; break; }
                if (g >= 2 && !ws_wait(bars, bars.bfree + bsel, (uint32_t)(((g - 2) >> 1) & 1))) { go = false; break; }
                unsigned char* Bhi = Bbuf + (size_t)bsel * 2 * BB;
                unsigned char* Blo = Bhi + BB;
                if (lane < NH) {
                    const unsigned char* tcol = Tbuf + (size_t)slot * TS + lane * TP;
                    for (int ks = warp; ks < nks; ks += WS_BUILDERS) {
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            float2 x[4];
#pragma unroll
                            for (int t = 0; t < 4; ++t) {
                                const int kk = 8 * ks + 4 * h + t;
                                x[t] = (lane < k && kk < r) ? *reinterpret_cast<const float2*>(tcol + kk * 8)
                                                            : make_float2(0.f, 0.f);
                            }
                            uint4 rh, rl, ih, il;
                            b_words(x, 0, rh, rl, ih, il);
                            const int ob = ks * KB;
                            *reinterpret_cast<uint4*>(Bhi + ob + kstep_off(lane, h)) = rh;
                            *reinterpret_cast<uint4*>(Blo + ob + kstep_off(lane, h)) = rl;
                            *reinterpret_cast<uint4*>(Bhi + ob + kstep_off(lane + NH, h)) = ih;
                            *reinterpret_cast<uint4*>(Blo + ob + kstep_off(lane + NH, h)) = il;
                        }
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(bars.bready + bsel));
            }
        }
        if (warp == 0 && lane == 0) bars.counts[2] = g;
    }
    if (ws_close(bars, tmem, 2 * N, ns)) {
        for (int w = blockIdx.x; w < nwork; w += gridDim.x)
            for (int e = tid; e < LM * k; e += blockDim.x) {
                const int jj = e / LM, rr = e - jj * LM;
                Y[(long long)jj * m + w * LM + rr] = make_float2(qnan(), qnan());
            }
        if (tid == 0) atomicAdd(&g_lr_tc_timeouts, 1);
    }
}

size_t partial_ws_smem(int NH, int rp, int k, int ns) {
    const size_t SAS = ((size_t)rp * 4 * LKC + 1023) & ~(size_t)1023;
    const size_t pre = ((size_t)ns * SAS + (size_t)ns * k * XPAD + 1023) & ~(size_t)1023;
    return pre + 4 * (size_t)(LKC / 8) * (2 * NH) * 32 + ws_bar_bytes(ns);
}
size_t apply_ws_smem(int NH, int r, int rp, int k, int ns) {
    const size_t SA = (size_t)(rp >> 3) * 4096, TS = ((size_t)k * (r * 8 + 16) + 127) & ~(size_t)127;
    const size_t pre = ((size_t)ns * SA + (size_t)ns * TS + 1023) & ~(size_t)1023;
    return pre + 4 * (size_t)(rp >> 3) * (2 * NH) * 32 + ws_bar_bytes(ns);
}

// persistent grid: every SM as many CTAs as its shared memory (1 KB of it
// reserved per CTA) and tensor memory (512 columns) hold, at most the work items
lsw_status persistent_grid(size_t smem, uint32_t tcols, int nwork, int& grid) {
    static std::atomic<int> sms{0}, smem_sm{0};
    if (sms.load() == 0) {
        int dev = 0, v = 0, w = 0;
        LSW_CUDA(cudaGetDevice(&dev));
        LSW_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
        LSW_CUDA(cudaDeviceGetAttribute(&w, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
        smem_sm.store(w);
        sms.store(v);
    }
    const int by_smem = (int)((size_t)smem_sm.load() / (smem + 1024));
    const int per = std::max(1, std::min(std::min(by_smem, (int)(512 / tcols)), 4));
    grid = std::max(1, std::min(nwork, sms.load() * per));
    return LSW_OK;
}

constexpr size_t kSmemCap = 200 * 1024;

template <int NH>
lsw_status partial_launch(const LrLevels<float2, uint32_t>& lv, int m, int r, int k, const float2* X, int swapA,
                          float2* P, cudaStream_t st) {
    static std::atomic<bool> attr{false};
    if (!attr.load()) {
        LSW_CUDA(cudaFuncSetAttribute(k_lr_partial_ws<NH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap));
        LSW_CUDA(cudaFuncSetAttribute(k_lr_partial_ws<NH>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
        attr.store(true);
    }
    // ring depth: 4 stages, 3 while the CTA does not fit two to an SM
    int ns = 4;
    if (partial_ws_smem(NH, lv.rp, k, ns) > 112 * 1024) ns = 3;
    const size_t smem = partial_ws_smem(NH, lv.rp, k, ns);
    int grid = 0;
    LSW_TRY(persistent_grid(smem, 4 * NH, lv.chunk0[lv.nlev], grid));
    k_lr_partial_ws<NH><<<grid, WS_THREADS, smem, st>>>(lv, m, r, k, X, swapA, P, ns);
    LSW_LAUNCH_CHECK();
    return LSW_OK;
}

template <int NH>
lsw_status apply_launch(const LrLevels<float2, uint32_t>& lv, int m, int r, int k, const float2* T, int swapC,
                        float2* Y, cudaStream_t st) {
    static std::atomic<bool> attr{false};
    if (!attr.load()) {
        LSW_CUDA(cudaFuncSetAttribute(k_lr_apply_ws<NH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap));
        LSW_CUDA(cudaFuncSetAttribute(k_lr_apply_ws<NH>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
        attr.store(true);
    }
    // ring depth: 3 stages (levels), 2 while the CTA does not fit two to an SM
    int ns = 3;
    if (apply_ws_smem(NH, r, lv.rp, k, ns) > 112 * 1024) ns = 2;
    const size_t smem = apply_ws_smem(NH, r, lv.rp, k, ns);
    int grid = 0;
    LSW_TRY(persistent_grid(smem, 4 * NH, m / LM, grid));
    k_lr_apply_ws<NH><<<grid, WS_THREADS, smem, st>>>(lv, m, r, k, T, swapC, Y, ns);
    LSW_LAUNCH_CHECK();
    return LSW_OK;
}

}  // namespace

bool lr_tc_fits(const LrLevels<float2, uint32_t>& lv, int m, int r, int k) {
    if (!tc_gemm_enabled() || k < 1 || k > 32 || r < 2 || (r & 1) || lv.rp < r || lv.rp > 64 || (lv.rp & 7) ||
        m % LM || lv.nlev < 1)
        return false;
    for (int q = 0; q < lv.nlev; ++q)
        if (lv.nb[q] % LM || lv.ch[q] % LKC || lv.flay[q] != FAC_TILE_P || lv.glay[q] != FAC_TILE_A) return false;
    return true;
}

lsw_status lr_partial_tc(const LrLevels<float2, uint32_t>& lv, int m, int r, int k, const float2* X, int swapA,
                         float2* P, cudaStream_t st) {
    return k <= 16 ? partial_launch<16>(lv, m, r, k, X, swapA, P, st) : partial_launch<32>(lv, m, r, k, X, swapA, P, st);
}

lsw_status lr_apply_tc(const LrLevels<float2, uint32_t>& lv, int m, int r, int k, const float2* T, int swapC,
                       float2* Y, cudaStream_t st) {
    return k <= 16 ? apply_launch<16>(lv, m, r, k, T, swapC, Y, st) : apply_launch<32>(lv, m, r, k, T, swapC, Y, st);
}

}  // namespace lsw
