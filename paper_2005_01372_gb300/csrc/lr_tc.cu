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
// into the B operand by the threads.  The CTAs are persistent: each walks its
// share of the work items (chunks, row tiles) as one stream of stages, with
// two TMEM accumulators so that an item's epilogue overlaps the next item's
// stages.  Every mbarrier wait is bounded; a wait that gives up writes NaN to
// the item's outputs, counts a timeout, drains the copies in flight (bounded)
// and frees the tensor memory before the CTA leaves.
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

// Pipeline state: a ring of ns stage buffers filled by bulk copies (one
// "full" mbarrier each), two B-operand buffers whose MMAs commit to one
// mbarrier each, one "accumulator ready" mbarrier per TMEM accumulator, the
// abort flag and the TMEM address.
struct Ring {
    uint64_t* full;
    uint64_t* mmab;
    uint64_t* accf;
    int* abort_flag;
    uint32_t* tslot;
    int* issued;
};
constexpr size_t ring_bytes(int ns) { return 8 * (size_t)ns + 16 + 16 + 16; }

__device__ __forceinline__ Ring ring_at(unsigned char* p, int ns) {
    Ring g;
    g.full = reinterpret_cast<uint64_t*>(p);
    g.mmab = g.full + ns;
    g.accf = g.mmab + 2;
    g.abort_flag = reinterpret_cast<int*>(g.accf + 2);
    g.tslot = reinterpret_cast<uint32_t*>(g.abort_flag + 1);
    g.issued = g.abort_flag + 2;
    return g;
}

__device__ __forceinline__ uint32_t ring_setup(const Ring& g, int ns, uint32_t tcols) {
    if (threadIdx.x == 0) {
        for (int i = 0; i < ns; ++i) mbar_init(smem_u32(g.full + i), 1);
        for (int i = 0; i < 2; ++i) {
            mbar_init(smem_u32(g.mmab + i), 1);
            mbar_init(smem_u32(g.accf + i), 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
        *g.abort_flag = 0;
    }
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(g.tslot)),
                     "r"(tcols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    return *g.tslot;
}

// Wait (bounded) for the copies issued but not consumed and for the last
// committed MMAs, then free the tensor memory.  All threads.
__device__ __forceinline__ void ring_close(const Ring& g, uint32_t tmem, uint32_t tcols, int ns, int consumed,
                                           int committed) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const int issued = *g.issued;
        for (int s = consumed; s < issued; ++s)
            if (!mbar_wait(smem_u32(g.full + s % ns), (s / ns) & 1)) *g.abort_flag = 1;
        if (committed > 0) {
            const int s = committed - 1;
            if (!mbar_wait(smem_u32(g.mmab + (s & 1)), (s >> 1) & 1)) *g.abort_flag = 1;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols));
}

// Accumulator b of 2 NH columns into d (lane = row), once its MMAs are done
// (the i-th use of accumulator b completes phase i of accf[b]).  All threads;
// returns false when the wait gave up.
template <int NH>
__device__ __forceinline__ bool acc_load(const Ring& g, uint32_t tmem, int li, float (&d)[2 * NH]) {
    const int b = li & 1;
    bool ok = mbar_wait(smem_u32(g.accf + b), (li >> 1) & 1);
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t taddr = tmem + (uint32_t)(b * 2 * NH) + ((uint32_t)((threadIdx.x >> 5) * 32) << 16);
#pragma unroll
    for (int col = 0; col < 2 * NH; col += 16) tmem_ld16(taddr + col, d + col);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    return ok;
}

// ------------------------------------------------------------- partials
// Work item w = chunk w of the level list (chunk0 numbering): CH rows of one
// level, in stages of LKC = 64 rows.  A stage's A'' (rows = the rp factor
// columns, K = the 64 rows: eight K-step tiles) is one contiguous copy of
// rp x 256 bytes of the tiled F; the MMA's rows rp..127 read whatever follows
// in shared memory and land in accumulator rows that are never read.  X's 64
// rows of each of the k columns are copied raw (512 B each) and become B''
// hi/lo in K-step tiles of 2 NH rows.  Warp 0 keeps ns stages in flight and
// refills the slot of stage g - 2, whose MMAs every thread has seen complete.
template <int NH>
__global__ void __launch_bounds__(128)
k_lr_partial_tc(LrLevels<float2, uint32_t> lv, int m, int r, int k, const float2* __restrict__ X, int swapA,
                float2* __restrict__ P, int ns) {
    constexpr int N = 2 * NH;
    constexpr uint32_t ID = idesc(1, LM, N);
    constexpr int KSP = LKC / 8;                       // K-steps per stage
    constexpr int KB = N * 32;                         // B'' bytes of one K-step
    constexpr int LBP = KSP * KB;                      // B'' bytes of a stage (hi or lo)
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
    const Ring g = ring_at(Bbuf + 4 * LBP, ns);
    const uint32_t tmem = ring_setup(g, ns, 2 * N);
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
    // producer cursor (warp 0)
    int iw = blockIdx.x, is = 0, issued = 0;
    Item ii{};
    if (iw < nwork) ii = item(iw);
    auto issue_next = [&]() {
        const int slot = issued % ns;
        const uint32_t fb = smem_u32(g.full + slot);
        const int nb = lv.nb[ii.q];
        const uint32_t* Asrc = lv.F[ii.q] + fac_index(FAC_TILE_P, nb, r, rp, ii.j, ii.o + is * LKC, 0);
        const float2* Xs = X + (long long)ii.src * nb + ii.o + is * LKC;
        if (lane == 0) mbar_expect_tx(fb, SA + (uint32_t)k * LKC * 8u);
        __syncwarp();
        if (lane == 0) bulk_g2s(smem_u32(Abuf + (size_t)slot * SAS), Asrc, SA, fb);
        if (lane < k)
            bulk_g2s(smem_u32(Xbuf + (size_t)slot * XS + lane * XPAD), Xs + (long long)lane * m, (uint32_t)LKC * 8u, fb);
        ++issued;
        if (++is == ii.S) {
            is = 0;
            iw += gridDim.x;
            if (iw < nwork) ii = item(iw);
        }
    };
    if (warp == 0)
        while (issued < ns && iw < nwork) issue_next();
    float d[N];
    auto epilogue = [&](int w, int l) {
        const bool ok = acc_load<NH>(g, tmem, l, d);
        if (tid < r) {
            float2* out = P + (long long)w * r * k;
#pragma unroll
            for (int jj = 0; jj < NH; ++jj)
                if (jj < k) out[(long long)jj * r + tid] = ok ? make_float2(d[jj], d[NH + jj]) : make_float2(qnan(), qnan());
        }
        if (!ok) *g.abort_flag = 1;
    };
    // consumer cursor (all threads)
    int cw = blockIdx.x, cs = 0, li = 0, gs = 0, committed = 0, pend = -1, pend_li = 0;
    Item ci{};
    if (cw < nwork) ci = item(cw);
    while (cw < nwork) {
        const int slot = gs % ns, bsel = gs & 1;
        if (!mbar_wait(smem_u32(g.full + slot), (gs / ns) & 1)) *g.abort_flag = 1;
        if (gs >= 2 && !mbar_wait(smem_u32(g.mmab + bsel), ((gs - 2) >> 1) & 1)) *g.abort_flag = 1;
        __syncthreads();
        if (*g.abort_flag) break;
        // B'' of the stage: thread (vector column lane, K-steps of warp)
        unsigned char* Bhi = Bbuf + (size_t)bsel * 2 * LBP;
        unsigned char* Blo = Bhi + LBP;
        if (lane < NH) {
            const float4* xs = reinterpret_cast<const float4*>(Xbuf + (size_t)slot * XS + lane * XPAD);
#pragma unroll
            for (int u = 0; u < KSP / 4; ++u) {
                const int ks = warp * (KSP / 4) + u;
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
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t a = smem_u32(Abuf + (size_t)slot * SAS), bh = smem_u32(Bhi), bl = smem_u32(Blo);
            const uint32_t dt = tmem + (uint32_t)((li & 1) * N);
#pragma unroll
            for (int ks = 0; ks < KSP; ++ks) {
                const uint64_t da = sdesc_sbo(a + ks * rp * 32, 256);
                mma_bf16(dt, da, sdesc_sbo(bh + ks * KB, 256), ID, (cs > 0 || ks > 0) ? 1u : 0u);
                mma_bf16(dt, da, sdesc_sbo(bl + ks * KB, 256), ID, 1u);
            }
            mma_commit(smem_u32(g.mmab + bsel));
            if (cs == ci.S - 1) mma_commit(smem_u32(g.accf + (li & 1)));
        }
        committed = gs + 1;
        if (warp == 0)
            while (iw < nwork && issued <= gs - 2 + ns) issue_next();
        if (pend >= 0) {
            epilogue(pend, pend_li);
            pend = -1;
        }
        ++gs;
        if (++cs == ci.S) {
            pend = cw;
            pend_li = li;
            ++li;
            cs = 0;
            cw += gridDim.x;
            if (cw < nwork) ci = item(cw);
        }
    }
    if (pend >= 0) epilogue(pend, pend_li);
    __syncthreads();
    const bool aborted = *g.abort_flag != 0;
    if (aborted) {
        // the items not finished get NaN
        for (int w = cw; w < nwork; w += gridDim.x)
            if (tid < r)
                for (int jj = 0; jj < k; ++jj) P[(long long)w * r * k + (long long)jj * r + tid] = make_float2(qnan(), qnan());
        if (tid == 0) atomicAdd(&g_lr_tc_timeouts, 1);
    }
    if (tid == 0) *g.issued = issued;   // warp 0's producer count
    ring_close(g, tmem, 2 * N, ns, gs, committed);
}

// ---------------------------------------------------------------- apply
// Work item = 128 rows of the node; one stage per level.  The tiled G holds
// the 128 rows' rp columns as rp / 8 contiguous 4 KB K-step tiles: one copy.
// The block's T (r x k, column-major) comes raw, a column at a time, and
// becomes B'' hi/lo (rp / 8 K-step tiles of 2 NH rows).  All levels
// accumulate in one TMEM accumulator, which the epilogue adds to Y.  Stages
// are large, so the ring is short: warp 0 refills the slot of stage g - 1
// once that stage's MMAs are done.
template <int NH>
__global__ void __launch_bounds__(128)
k_lr_apply_tc(LrLevels<float2, uint32_t> lv, int m, int r, int k, const float2* __restrict__ T, int swapC,
              float2* __restrict__ Y, int ns) {
    constexpr int N = 2 * NH;
    constexpr uint32_t ID = idesc(1, LM, N);
    extern __shared__ __align__(1024) unsigned char sm[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwork = m / LM;
    const long long nout = (long long)r * k;
    const int rp = lv.rp, nks = rp >> 3;
    const uint32_t SA = (uint32_t)nks * 4096u;               // A bytes per level
    const int TP = r * 8 + 16;                               // smem stride of a raw T column
    const int TS = (k * TP + 127) & ~127;
    const int KB = N * 32;                                   // B'' bytes of one K-step
    const int BB = nks * KB;                                 // B'' bytes of a stage (hi or lo)
    unsigned char* Abuf = sm;
    unsigned char* Tbuf = sm + (size_t)ns * SA;
    unsigned char* Bbuf = sm + (((size_t)ns * SA + (size_t)ns * TS + 1023) & ~(size_t)1023);
    const Ring g = ring_at(Bbuf + 4 * BB, ns);
    const uint32_t tmem = ring_setup(g, ns, 2 * N);
    const int S = lv.nlev;
    // producer cursor (warp 0): item iw, level is
    int iw = blockIdx.x, is = 0, issued = 0;
    auto issue_next = [&]() {
        const int slot = issued % ns;
        const int nb = lv.nb[is];
        const int i0 = iw * LM;
        const int b = i0 / nb, o = i0 - b * nb;
        const int bb = swapC ? (b ^ 1) : b;
        const uint32_t fb = smem_u32(g.full + slot);
        if (lane == 0) mbar_expect_tx(fb, SA + (uint32_t)k * r * 8u);
        __syncwarp();
        if (lane == 0)
            bulk_g2s(smem_u32(Abuf + (size_t)slot * SA), lv.G[is] + fac_index(FAC_TILE_A, nb, r, rp, bb, o, 0), SA, fb);
        if (lane < k)
            bulk_g2s(smem_u32(Tbuf + (size_t)slot * TS + lane * TP), T + (lv.t0[is] + bb) * nout + (long long)lane * r,
                     (uint32_t)r * 8u, fb);
        ++issued;
        if (++is == S) {
            is = 0;
            iw += gridDim.x;
        }
    };
    if (warp == 0)
        while (issued < ns && iw < nwork) issue_next();
    float d[N];
    auto epilogue = [&](int w, int l) {
        const bool ok = acc_load<NH>(g, tmem, l, d);
        const int row = w * LM + tid;
#pragma unroll
        for (int jj = 0; jj < NH; ++jj) {
            if (jj >= k) continue;
            float2* y = Y + (long long)jj * m + row;
            float2 v = *y;
            v = ok ? make_float2(v.x + d[jj], v.y + d[NH + jj]) : make_float2(qnan(), qnan());
            *y = v;
        }
        if (!ok) *g.abort_flag = 1;
    };
    int cw = blockIdx.x, cs = 0, li = 0, gs = 0, committed = 0, pend = -1, pend_li = 0;
    while (cw < nwork) {
        const int slot = gs % ns, bsel = gs & 1;
        if (!mbar_wait(smem_u32(g.full + slot), (gs / ns) & 1)) *g.abort_flag = 1;
        if (gs >= 2 && !mbar_wait(smem_u32(g.mmab + bsel), ((gs - 2) >> 1) & 1)) *g.abort_flag = 1;
        __syncthreads();
        if (*g.abort_flag) break;
        unsigned char* Bhi = Bbuf + (size_t)bsel * 2 * BB;
        unsigned char* Blo = Bhi + BB;
        if (lane < NH) {
            const unsigned char* tcol = Tbuf + (size_t)slot * TS + lane * TP;
            for (int ks = warp; ks < nks; ks += 4) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    // complex K 8 ks + 4 h .. + 3 of column lane (beyond r: zero)
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
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t a = smem_u32(Abuf + (size_t)slot * SA), bh = smem_u32(Bhi), bl = smem_u32(Blo);
            const uint32_t dt = tmem + (uint32_t)((li & 1) * N);
            for (int ks = 0; ks < nks; ++ks) {
                const uint64_t da = sdesc_sbo(a + ks * 4096, 256);
                mma_bf16(dt, da, sdesc_sbo(bh + ks * KB, 256), ID, (cs > 0 || ks > 0) ? 1u : 0u);
                mma_bf16(dt, da, sdesc_sbo(bl + ks * KB, 256), ID, 1u);
            }
            mma_commit(smem_u32(g.mmab + bsel));
            if (cs == S - 1) mma_commit(smem_u32(g.accf + (li & 1)));
        }
        committed = gs + 1;
        if (warp == 0 && gs >= 1 && iw < nwork && issued <= gs - 1 + ns) {
            if (mbar_wait(smem_u32(g.mmab + ((gs - 1) & 1)), ((gs - 1) >> 1) & 1))
                issue_next();
            else if (lane == 0)
                *g.abort_flag = 1;
        }
        if (pend >= 0) {
            epilogue(pend, pend_li);
            pend = -1;
        }
        ++gs;
        if (++cs == S) {
            pend = cw;
            pend_li = li;
            ++li;
            cs = 0;
            cw += gridDim.x;
        }
    }
    if (pend >= 0) epilogue(pend, pend_li);
    __syncthreads();
    if (*g.abort_flag) {
        for (int w = cw; w < nwork; w += gridDim.x)
            for (int jj = 0; jj < k; ++jj) Y[(long long)jj * m + w * LM + tid] = make_float2(qnan(), qnan());
        if (tid == 0) atomicAdd(&g_lr_tc_timeouts, 1);
    }
    if (tid == 0) *g.issued = issued;   // warp 0's producer count
    ring_close(g, tmem, 2 * N, ns, gs, committed);
}

// shared memory of the two kernels for a ring of ns stages
size_t partial_smem(int NH, int rp, int k, int ns) {
    const size_t SAS = ((size_t)rp * 4 * LKC + 1023) & ~(size_t)1023;
    const size_t pre = ((size_t)ns * SAS + (size_t)ns * k * XPAD + 1023) & ~(size_t)1023;
    return pre + 4 * (size_t)(LKC / 8) * (2 * NH) * 32 + ring_bytes(ns);
}
size_t apply_smem(int NH, int r, int rp, int k, int ns) {
    const size_t SA = (size_t)(rp >> 3) * 4096, TS = ((size_t)k * (r * 8 + 16) + 127) & ~(size_t)127;
    const size_t pre = ((size_t)ns * SA + (size_t)ns * TS + 1023) & ~(size_t)1023;
    return pre + 4 * (size_t)(rp >> 3) * (2 * NH) * 32 + ring_bytes(ns);
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
        LSW_CUDA(cudaFuncSetAttribute(k_lr_partial_tc<NH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap));
        LSW_CUDA(cudaFuncSetAttribute(k_lr_partial_tc<NH>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
        attr.store(true);
    }
    // ring depth: 4 stages, 3 while the CTA does not fit two to an SM
    int ns = 4;
    if (partial_smem(NH, lv.rp, k, ns) > 112 * 1024) ns = 3;
    const size_t smem = partial_smem(NH, lv.rp, k, ns);
    int grid = 0;
    LSW_TRY(persistent_grid(smem, 4 * NH, lv.chunk0[lv.nlev], grid));
    k_lr_partial_tc<NH><<<grid, 128, smem, st>>>(lv, m, r, k, X, swapA, P, ns);
    LSW_LAUNCH_CHECK();
    return LSW_OK;
}

template <int NH>
lsw_status apply_launch(const LrLevels<float2, uint32_t>& lv, int m, int r, int k, const float2* T, int swapC,
                        float2* Y, cudaStream_t st) {
    static std::atomic<bool> attr{false};
    if (!attr.load()) {
        LSW_CUDA(cudaFuncSetAttribute(k_lr_apply_tc<NH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap));
        LSW_CUDA(cudaFuncSetAttribute(k_lr_apply_tc<NH>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
        attr.store(true);
    }
    // ring depth: 3 stages (levels), 2 while the CTA does not fit two to an SM
    int ns = 3;
    if (apply_smem(NH, r, lv.rp, k, ns) > 112 * 1024) ns = 2;
    const size_t smem = apply_smem(NH, r, lv.rp, k, ns);
    int grid = 0;
    LSW_TRY(persistent_grid(smem, 4 * NH, m / LM, grid));
    k_lr_apply_tc<NH><<<grid, 128, smem, st>>>(lv, m, r, k, T, swapC, Y, ns);
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
