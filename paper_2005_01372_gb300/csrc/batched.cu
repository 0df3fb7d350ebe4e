// Many (grid, frequency) problems in one call, and the measured choice of
// FFT pass variant per size.
//
// The paper's method serves every source of one (grid, frequency) with one
// preconditioner (Sec. 3: "the same preconditioner could be used for all
// sources").  lsw_solve_batched takes many such problems: each gets its own
// Green handle, contrast, sources and preconditioner; problems run
// concurrently from host worker threads, each driving its own CUDA stream
// (and its own fork pool), so that latency-bound builds of different
// problems overlap on the GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <thread>
#include <vector>

#include "lsw_internal.cuh"

namespace lsw {
int op_variant(int pz, int px, int rsize);
void op_force_variant(int v);
void op_set_variant(int pz, int px, int rsize, int v);
}  // namespace lsw

using namespace lsw;

namespace {
template <typename C>
__global__ void k_sub(const C* __restrict__ a, const C* __restrict__ b, C* __restrict__ d, long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        C v = a[e];
        v.x -= b[e].x;
        v.y -= b[e].y;
        d[e] = v;
    }
}
}  // namespace

extern "C" {

lsw_status lsw_autotune(const lsw_green* g, int prec, int nbatch, void* stream, int* variant, float* ms3) {
    if (!g || nbatch <= 0 || (prec != LSW_C128 && prec != LSW_C64)) return LSW_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const long long n = (long long)g->nz * g->nx;
    const size_t elem = prec == LSW_C128 ? sizeof(double2) : sizeof(float2);
    DevBuf u, y, y0, work, chi, w2, w3, nrm;
    LSW_TRY(u.alloc(elem * n * nbatch, st));
    LSW_TRY(y.alloc(elem * n * nbatch, st));
    LSW_TRY(y0.alloc(elem * n * nbatch, st));
    LSW_TRY(work.alloc(elem * 2 * n * nbatch, st));
    LSW_TRY(chi.alloc(sizeof(double) * n, st));
    LSW_TRY(w2.alloc(sizeof(uint32_t) * nbatch, st));
    LSW_TRY(w3.alloc(sizeof(uint32_t) * nbatch, st));
    LSW_TRY(nrm.alloc(sizeof(double) * 2, st));
    // a seeded Gaussian field and chi = 0.001 everywhere: every variant must
    // reproduce variant 0's result before it may be chosen
    LSW_CUDA(cudaMemsetAsync(w2.p, 0, sizeof(uint32_t) * nbatch, st));
    LSW_CUDA(cudaMemsetAsync(w3.p, 0, sizeof(uint32_t) * nbatch, st));
    if (prec == LSW_C128)
        LSW_TRY(gaussian_fill<double>(u.as<double2>(), (int)n, 1, n, nbatch, 12345, w2.as<uint32_t>(), w3.as<uint32_t>(), st));
    else
        LSW_TRY(gaussian_fill<float>(u.as<float2>(), (int)n, 1, n, nbatch, 12345, w2.as<uint32_t>(), w3.as<uint32_t>(), st));
    {
        std::vector<double> c(n, 1e-3);
        LSW_CUDA(cudaMemcpyAsync(chi.p, c.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
        LSW_CUDA(cudaStreamSynchronize(st));
    }
    OpGeom geo{g->nz, g->nx, chi.as<double>(), g->nz, nullptr, 1};
    cudaEvent_t e0, e1;
    LSW_CUDA(cudaEventCreate(&e0));
    LSW_CUDA(cudaEventCreate(&e1));
    float best = 0;
    int bestv = 0;
    lsw_status rc = LSW_OK;
    for (int v = 0; v < 3 && rc == LSW_OK; ++v) {
        op_force_variant(v);
        auto run = [&]() -> lsw_status {
            if (prec == LSW_C128)
                return op_apply<double>(g, g->full, geo, LSW_OP_PLAIN, u.as<double2>(), nullptr, y.as<double2>(), nbatch,
                                        work.as<double2>(), st);
            return op_apply<float>(g, g->full, geo, LSW_OP_PLAIN, u.as<float2>(), nullptr, y.as<float2>(), nbatch,
                                   work.as<float2>(), st);
        };
        float ms = -1;
        lsw_status s = LSW_OK;
        for (int w = 0; w < 3 && s == LSW_OK; ++w) s = run();
        if (s == LSW_OK) {
            // check against variant 0: relative 2-norm difference
            if (v == 0) {
                LSW_CUDA(cudaMemcpyAsync(y0.p, y.p, elem * n * nbatch, cudaMemcpyDeviceToDevice, st));
            } else {
                double h[2] = {0, 0};
                if (prec == LSW_C128) {
                    k_sub<double2><<<1024, 256, 0, st>>>(y.as<double2>(), y0.as<double2>(), y.as<double2>(), n * nbatch);
                    LSW_LAUNCH_CHECK();
                    LSW_TRY(norms2<double>(y.as<double2>(), n * nbatch, 1, nrm.as<double>(), st));
                    LSW_TRY(norms2<double>(y0.as<double2>(), n * nbatch, 1, nrm.as<double>() + 1, st));
                } else {
                    k_sub<float2><<<1024, 256, 0, st>>>(y.as<float2>(), y0.as<float2>(), y.as<float2>(), n * nbatch);
                    LSW_LAUNCH_CHECK();
                    LSW_TRY(norms2<float>(y.as<float2>(), n * nbatch, 1, nrm.as<double>(), st));
                    LSW_TRY(norms2<float>(y0.as<float2>(), n * nbatch, 1, nrm.as<double>() + 1, st));
                }
                LSW_CUDA(cudaMemcpyAsync(h, nrm.p, sizeof h, cudaMemcpyDeviceToHost, st));
                LSW_CUDA(cudaStreamSynchronize(st));
                const double tolv = prec == LSW_C128 ? 1e-12 : 1e-5;
                if (!(h[0] <= tolv * tolv * h[1])) s = LSW_ERR_NUMERIC;
            }
        }
        if (s == LSW_OK) {
            cudaEventRecord(e0, st);
            for (int r = 0; r < 10 && s == LSW_OK; ++r) s = run();
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
            ms /= 10;
        }
        if (s != LSW_OK && s != LSW_ERR_UNSUPPORTED_SIZE && s != LSW_ERR_NUMERIC) rc = s;
        if (ms3) ms3[v] = s == LSW_OK ? ms : (s == LSW_ERR_NUMERIC ? -2.0f : -1.0f);
        if (s == LSW_OK && (best == 0 || ms < best)) {
            best = ms;
            bestv = v;
        }
    }
    op_force_variant(-1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != LSW_OK) return rc;
    op_set_variant(2 * g->nz, 2 * g->nx, prec == LSW_C128 ? 8 : 4, bestv);
    // a variant whose result differed from variant 0 reports -2 in ms3
    if (variant) *variant = bestv;
    return LSW_OK;
}

lsw_status lsw_solve_batched(const lsw_problem* probs, int nprob, const lsw_hparams* hp, const lsw_solve_params* sp,
                             int max_concurrent, lsw_solve_info* info, void* stream) {
    if (!probs || nprob < 0 || !sp || !info) return LSW_ERR_INVALID_ARG;
    if (nprob == 0) return LSW_OK;
    for (int i = 0; i < nprob; ++i)
        if (!probs[i].velocity || !probs[i].sources || probs[i].nsrc <= 0 || !probs[i].u) return LSW_ERR_INVALID_ARG;
    // inputs may come from work on the caller's stream
    LSW_CUDA(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)));
    std::vector<int> offset(nprob + 1, 0);
    for (int i = 0; i < nprob; ++i) offset[i + 1] = offset[i] + probs[i].nsrc;
    std::vector<lsw_status> status(nprob, LSW_OK);
    int dev = 0;
    LSW_CUDA(cudaGetDevice(&dev));
    const int upcast = sp->prec == LSW_C64 ? LSW_C64 : LSW_C128;
    const size_t elem = upcast == LSW_C128 ? sizeof(double2) : sizeof(float2);
    std::atomic<int> next{0};
    auto worker = [&](int slot) {
        cudaSetDevice(dev);
        set_worker_slot(slot);
        cudaStream_t s;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            for (int i; (i = next++) < nprob;) status[i] = LSW_ERR_CUDA;
            return;
        }
        for (int i; (i = next++) < nprob;) {
            const lsw_problem& p = probs[i];
            lsw_green* g = nullptr;
            lsw_hmatrix* h = nullptr;
            lsw_status st = lsw_build_green(&p.grid, s, &g);
            const long long n = (long long)p.grid.nz * p.grid.nx;
            void* chi = nullptr;
            void* u0 = nullptr;
            if (st == LSW_OK && cudaMallocAsync(&chi, sizeof(double) * n, s) != cudaSuccess) st = LSW_ERR_OOM;
            if (st == LSW_OK && cudaMallocAsync(&u0, elem * n * p.nsrc, s) != cudaSuccess) st = LSW_ERR_OOM;
            if (st == LSW_OK) st = lsw_contrast(g, p.velocity, (double*)chi, s);
            if (st == LSW_OK) st = lsw_point_sources(g, p.sources, p.nsrc, upcast, u0, s);
            // rank adaptation: a problem that leaves a source unconverged is
            // rebuilt with twice the rank (at most rank_max) and solved again
            lsw_hparams hpl;
            if (hp) hpl = *hp;
            for (;;) {
                if (st == LSW_OK && hp) st = lsw_build_hmatrix(g, (const double*)chi, &hpl, s, &h);
                if (st != LSW_OK) break;
                st = lsw_solve_series(g, (const double*)chi, h, u0, p.u, p.nsrc, sp, info + offset[i], s);
                // the sketches take at most 64 probes: rank + oversample <= 64
                const int next = hp ? std::min({hpl.rank_max, 2 * hpl.rank, 64 - hpl.oversample}) : 0;
                const bool retry = hp && hpl.kind == LSW_H_HODLR && next > hpl.rank &&
                                   (st == LSW_ERR_NOT_CONVERGED || st == LSW_ERR_DIVERGED ||
                                    st == LSW_ERR_NUMERIC);
                if (!retry) break;
                lsw_destroy_hmatrix(h);
                h = nullptr;
                hpl.rank = next;
                st = LSW_OK;
            }
            if (h) lsw_destroy_hmatrix(h);
            if (chi) cudaFreeAsync(chi, s);
            if (u0) cudaFreeAsync(u0, s);
            cudaStreamSynchronize(s);
            if (g) lsw_destroy_green(g);
            status[i] = st;
        }
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
        set_worker_slot(0);
    };
    const int nw = std::max(1, std::min({max_concurrent > 0 ? max_concurrent : 4, nprob, 7}));
    std::vector<std::thread> pool;
    for (int w = 0; w < nw; ++w) pool.emplace_back(worker, w + 1);
    for (auto& t : pool) t.join();
    for (int i = 0; i < nprob; ++i)
        if (status[i] != LSW_OK) return status[i];
    return LSW_OK;
}

lsw_status lsw_sweep_next_rank(const lsw_sweep_policy* pol, int32_t rank, int32_t solve_status,
                               int32_t max_iterations, int32_t* next_rank, int32_t* rebuild) {
    if (!pol || !next_rank || !rebuild || rank < 1 || pol->rank0 < 1 || pol->rank_step < 1 ||
        pol->rank_max < pol->rank0 || pol->raise_iters < 0)
        return LSW_ERR_INVALID_ARG;
    const int32_t grown = std::min(rank + pol->rank_step, pol->rank_max);
    if (solve_status != LSW_OK) {
        // not converged within the limit: a larger rank, from psi0 again
        *rebuild = grown > rank ? 1 : 0;
        *next_rank = *rebuild ? grown : rank;
    } else {
        // converged, but slowly: the next frequency starts higher
        *rebuild = 0;
        *next_rank = max_iterations > pol->raise_iters ? std::max(grown, rank) : rank;
    }
    return LSW_OK;
}

lsw_status lsw_solve_sweep(const lsw_grid* grid, const double* velocity, const double* freqs_hz, int nfreq,
                           const int32_t* sources, int nsrc, const lsw_hparams* hp, const lsw_sweep_policy* pol,
                           const lsw_solve_params* sp, void* u, lsw_sweep_info* info, lsw_solve_info* sinfo,
                           void* stream) {
    if (!grid || !velocity || nfreq < 0 || (nfreq > 0 && !freqs_hz) || !sources || nsrc <= 0 || !hp || !pol || !sp ||
        !u || !info)
        return LSW_ERR_INVALID_ARG;
    if (hp->kind != LSW_H_HODLR || pol->rank0 < 1 || pol->rank_step < 1 || pol->rank_max < pol->rank0 ||
        pol->raise_iters < 0 || hp->oversample < 0 || pol->rank_max + hp->oversample > 64)
        return LSW_ERR_INVALID_ARG;
    if (nfreq == 0) return LSW_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const long long n = (long long)grid->nz * grid->nx;
    const int upcast = sp->prec == LSW_C64 ? LSW_C64 : LSW_C128;
    const size_t elem = upcast == LSW_C128 ? sizeof(double2) : sizeof(float2);
    DevBuf chi, u0;
    LSW_TRY(chi.alloc(sizeof(double) * n, s));
    LSW_TRY(u0.alloc(elem * n * nsrc, s));
    std::vector<lsw_solve_info> si(nsrc);
    lsw_hparams hpl = *hp;
    hpl.rank_max = 0;
    int32_t rank = pol->rank0;
    lsw_status first_fail = LSW_OK;
    for (int f = 0; f < nfreq; ++f) {
        lsw_grid gf = *grid;
        gf.freq_hz = freqs_hz[f];
        lsw_green* g = nullptr;
        LSW_TRY(lsw_build_green(&gf, s, &g));
        struct GreenGuard {
            lsw_green* g;
            cudaStream_t s;
            ~GreenGuard() {
                cudaStreamSynchronize(s);
                lsw_destroy_green(g);
            }
        } guard{g, s};
        LSW_TRY(lsw_contrast(g, velocity, chi.as<double>(), s));
        LSW_TRY(lsw_point_sources(g, sources, nsrc, upcast, u0.p, s));
        void* uf = static_cast<char*>(u) + (size_t)f * nsrc * n * elem;
        lsw_sweep_info& inf = info[f];
        inf = lsw_sweep_info{};
        inf.freq_hz = freqs_hz[f];
        lsw_status st;
        for (;;) {
            hpl.rank = rank;
            lsw_hmatrix* h = nullptr;
            LSW_TRY(lsw_build_hmatrix(g, chi.as<double>(), &hpl, s, &h));
            ++inf.builds;
            st = lsw_solve_series(g, chi.as<double>(), h, u0.p, uf, nsrc, sp, si.data(), s);
            lsw_destroy_hmatrix(h);
            if (st != LSW_OK && st != LSW_ERR_NOT_CONVERGED && st != LSW_ERR_DIVERGED && st != LSW_ERR_NUMERIC)
                return st;
            int32_t maxit = 0, conv = 0;
            double maxres = 0;
            for (const auto& x : si) {
                maxit = std::max(maxit, x.iterations);
                conv += x.status == LSW_OK;
                maxres = std::max(maxres, x.rel_residual);
            }
            int32_t next = rank, rebuild = 0;
            LSW_TRY(lsw_sweep_next_rank(pol, rank, st, maxit, &next, &rebuild));
            inf.rank = rank;
            inf.converged = conv;
            inf.max_iterations = maxit;
            inf.max_rel_residual = maxres;
            inf.status = st;
            inf.next_rank = next;
            rank = next;
            if (!rebuild) break;
        }
        if (sinfo)
            for (int i = 0; i < nsrc; ++i) sinfo[(size_t)f * nsrc + i] = si[i];
        if (st != LSW_OK && first_fail == LSW_OK) first_fail = st;
    }
    LSW_CUDA(cudaStreamSynchronize(s));
    return first_fail;
}

}  // extern "C"
