// Solvers for (I - G0 V) psi = psi0 (Eq. 5): the preconditioned scattering
// series (Eq. 11; Born series when H is absent, Sec. 2.2), flexible GMRES
// with H as right preconditioner (the Krylov comparison of Sec. 3.2), and
// mixed-precision iterative refinement around either (FP64 residual, FP32
// corrections).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "lsw_internal.cuh"

struct lsw_hmatrix;

namespace lsw {

template <typename R>
lsw_status apply_h(const lsw_hmatrix* h, const typename Cx<R>::T* x, typename Cx<R>::T* y, int nb, cudaStream_t st);
int hmatrix_prec(const lsw_hmatrix* h);
lsw_status fno_apply_precond(const lsw_fno* f, const lsw_green* g, const double* chi, const void* v, void* z, int nb,
                             int prec, cudaStream_t st);
bool fno_matches(const lsw_fno* f, const lsw_green* g);

// The learned right preconditioner of a solve and whether it has been
// dropped for H.
struct Learned {
    const lsw_fno* fno = nullptr;
    bool off = false;
};

namespace {

int gridn(long long n, int bs = 256) {
    long long g = (n + bs - 1) / bs;
    return (int)std::max<long long>(1, std::min<long long>(g, 152LL * 32));
}

struct SrcInfo {
    int iters = 0;
    int status = LSW_ERR_NOT_CONVERGED;
    double rel = INFINITY;
};

// u_s += alpha * t_s for sources with active[s]
template <typename C, typename R>
__global__ void k_masked_axpy(C* __restrict__ u, const C* __restrict__ t, const int* __restrict__ active, long long n,
                              int nb, R alpha) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n * nb; e += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(e / n);
        if (!active[s]) continue;
        C a = u[e];
        const C b = t[e];
        a.x += alpha * b.x;
        a.y += alpha * b.y;
        u[e] = a;
    }
}

// dst_s = scale_s * src_s  (any precisions)
template <typename Cs, typename Cd>
__global__ void k_scale_cast(const Cs* __restrict__ src, Cd* __restrict__ dst, const double* __restrict__ scale,
                             long long n, int nb) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n * nb; e += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(e / n);
        const double a = scale ? scale[s] : 1.0;
        const Cs v = src[e];
        Cd o;
        o.x = (double)v.x * a;
        o.y = (double)v.y * a;
        dst[e] = o;
    }
}

// u64_s += d_s (cast up) for active sources
template <typename Cd>
__global__ void k_add_up(double2* __restrict__ u, const Cd* __restrict__ d, const int* __restrict__ active, long long n,
                         int nb) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n * nb; e += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(e / n);
        if (!active[s]) continue;
        const Cd v = d[e];
        u[e].x += (double)v.x;
        u[e].y += (double)v.y;
    }
}

template <typename T>
lsw_status up(DevBuf& b, const std::vector<T>& v, cudaStream_t st) {
    if (!b.p) LSW_TRY(b.alloc(sizeof(T) * std::max<size_t>(1, v.size()), st));
    LSW_CUDA(cudaMemcpyAsync(b.p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st));
    return LSW_OK;
}

// squared norms of nb fields to the host (synchronises)
template <typename R>
lsw_status host_norms(const typename Cx<R>::T* x, long long n, int nb, DevBuf& dn, std::vector<double>& out,
                      cudaStream_t st) {
    if (!dn.p) LSW_TRY(dn.alloc(sizeof(double) * nb, st));
    LSW_TRY(norms2<R>(x, n, nb, dn.as<double>(), st));
    out.resize(nb);
    LSW_CUDA(cudaMemcpyAsync(out.data(), dn.p, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
    LSW_CUDA(cudaStreamSynchronize(st));
    return LSW_OK;
}

template <typename R>
lsw_status op_full(const lsw_green* g, const double* chi, int mode, const typename Cx<R>::T* u,
                   const typename Cx<R>::T* u0, typename Cx<R>::T* y, int nb, DevBuf& work, cudaStream_t st) {
    typedef typename Cx<R>::T C;
    const long long n = (long long)g->nz * g->nx;
    if (!work.p) LSW_TRY(work.alloc(sizeof(C) * 2 * n * nb, st));
    OpGeom geo{g->nz, g->nx, chi, g->nz, nullptr, 1};
    return op_apply<R>(g, g->full, geo, mode, u, u0, y, nb, work.as<C>(), st);
}

// ----------------------------------------------------------------- series
// Eq. 11 for nb sources in precision R; per source: iterations, status and
// the relative residual of the returned field (in precision R).
template <typename R>
lsw_status series_run(const lsw_green* g, const double* chi, const lsw_hmatrix* h, const typename Cx<R>::T* u0,
                      typename Cx<R>::T* u, int nb, int max_iter, double tol, std::vector<SrcInfo>& info,
                      cudaStream_t st) {
    typedef typename Cx<R>::T C;
    const long long n = (long long)g->nz * g->nx;
    DevBuf a, t, work, dn, act;
    LSW_TRY(a.alloc(sizeof(C) * n * nb, st));
    LSW_TRY(t.alloc(sizeof(C) * n * nb, st));
    std::vector<double> n0, na;
    LSW_TRY(host_norms<R>(u0, n, nb, dn, n0, st));
    info.assign(nb, SrcInfo());
    std::vector<int> active(nb, 1);
    std::vector<double> best(nb, INFINITY);
    // psi_0 = H psi0 (Eq. 9 with phi_0 = H psi0), or psi0 for Born
    if (h) LSW_TRY(apply_h<R>(h, u0, u, nb, st));
    else LSW_CUDA(cudaMemcpyAsync(u, u0, sizeof(C) * n * nb, cudaMemcpyDeviceToDevice, st));
    for (int s = 0; s < nb; ++s)
        if (!(n0[s] > 0)) {     // zero right-hand side: psi = 0
            active[s] = 0;
            info[s].status = LSW_OK;
            info[s].rel = 0;
            LSW_CUDA(cudaMemsetAsync(u + s * n, 0, sizeof(C) * n, st));
        }
    for (int it = 0;; ++it) {
        // a = psi - G0 V psi - psi0   (Eq. 13)
        LSW_TRY(op_full<R>(g, chi, LSW_OP_RESIDUAL, u, u0, a.as<C>(), nb, work, st));
        LSW_TRY(host_norms<R>(a.as<C>(), n, nb, dn, na, st));
        int left = 0;
        for (int s = 0; s < nb; ++s) {
            if (!active[s]) continue;
            const double rel = std::sqrt(na[s] / n0[s]);
            info[s].iters = it;
            info[s].rel = rel;
            if (!std::isfinite(rel)) { info[s].status = LSW_ERR_NUMERIC; active[s] = 0; continue; }
            if (rel <= tol) { info[s].status = LSW_OK; active[s] = 0; continue; }
            best[s] = std::min(best[s], rel);
            if (rel > 1e3 * best[s]) { info[s].status = LSW_ERR_DIVERGED; active[s] = 0; continue; }
            if (it == max_iter) { info[s].status = LSW_ERR_NOT_CONVERGED; active[s] = 0; continue; }
            ++left;
        }
        if (!left) break;
        // psi <- psi - H a
        if (h) LSW_TRY(apply_h<R>(h, a.as<C>(), t.as<C>(), nb, st));
        LSW_TRY(up(act, active, st));
        k_masked_axpy<C, R><<<gridn(n * nb), 256, 0, st>>>(u, h ? t.as<C>() : a.as<C>(), act.as<int>(), n, nb, (R)-1);
        LSW_LAUNCH_CHECK();
    }
    return LSW_OK;
}

// ------------------------------------------------------------- step graph
// The Arnoldi step's fixed-buffer work (v_j -> z_j = H v_j -> w = A z_j) as
// one CUDA graph: the first run() eagerly runs it, the second captures it on
// a stream of its own (the caller's may be the legacy default stream, which
// cannot capture) and every run() from then on replays it there, ordered
// after and before the caller's stream by two events: one launch instead of
// a dozen.  Any capture or instantiation failure, a caller that is itself
// capturing, or graphs switched off keeps the eager path.  Replays add the
// captured kernels to the launch counter.
struct StepGraph {
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cs = nullptr;                 // capture and replay stream (the
    cudaEvent_t in = nullptr, out = nullptr;   // caller's may be the legacy one)
    int runs = 0;
    bool failed = false;
    long long launches = 0;
    std::vector<TimedSpan> spans;              // timer events inside the graph
    bool unharvested = false;
    ~StepGraph() {
        if (unharvested) timer_harvest(spans);
        timer_release(spans);
        if (exec) cudaGraphExecDestroy(exec);
        if (in) cudaEventDestroy(in);
        if (out) cudaEventDestroy(out);
        if (cs) cudaStreamDestroy(cs);
    }
    // body(stream) enqueues the step on the given stream
    template <typename F>
    lsw_status run(cudaStream_t st, F&& body) {
        ++runs;
        if (exec) return replay(st);
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        if (failed || runs < 2 || !graphs_enabled() || cudaStreamIsCapturing(st, &cap) != cudaSuccess ||
            cap != cudaStreamCaptureStatusNone)
            return body(st);
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&in, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&out, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            failed = true;
            return body(st);
        }
        const unsigned long long l0 = launch_counter();
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
            cudaGetLastError();
            failed = true;
            return body(st);
        }
        const lsw_status s = body(cs);
        cudaGraph_t gr = nullptr;
        const cudaError_t e = cudaStreamEndCapture(cs, &gr);
        launches = (long long)(launch_counter() - l0);
        spans = timer_take_captured();
        if (s == LSW_OK && e == cudaSuccess && gr && cudaGraphInstantiate(&exec, gr, 0) != cudaSuccess) exec = nullptr;
        if (gr) cudaGraphDestroy(gr);
        cudaGetLastError();
        if (!exec) {
            // nothing captured ran: take back its count and run it eagerly
            timer_release(spans);
            failed = true;
            count_launches(-launches);
            return body(st);
        }
        count_launches(-launches);              // counted again by the replay
        return replay(st);
    }

  private:
    lsw_status replay(cudaStream_t st) {
        // the previous replay's timer spans (its work is ordered before this one)
        if (unharvested) timer_harvest(spans);
        unharvested = !spans.empty();
        LSW_CUDA(cudaEventRecord(in, st));
        LSW_CUDA(cudaStreamWaitEvent(cs, in, 0));
        LSW_CUDA(cudaGraphLaunch(exec, cs));
        LSW_CUDA(cudaEventRecord(out, cs));
        LSW_CUDA(cudaStreamWaitEvent(st, out, 0));
        count_launches(launches);
        count_graph_replay();
        return LSW_OK;
    }
};

// ----------------------------------------------------------------- FGMRES
// Flexible GMRES(m) for nb independent sources in lockstep, from x = 0, with
// H (or the learned network while it is on) as right preconditioner; Arnoldi
// by classical Gram-Schmidt applied twice, the small least-squares problems
// by Givens rotations on the host in FP64.  While the network preconditions,
// every kProbe iterations of a cycle each active source's residual estimate
// must have dropped below kProbeRatio times its value kProbe iterations
// earlier; otherwise the cycle ends there and the network is off for the
// rest of the solve.  A cycle cut at its first probe does not update x (its
// directions are what failed); a later one does, with directions whose
// least-squares pivot is negligible against the largest left out.
constexpr int kProbe = 5;
constexpr double kProbeRatio = 0.5;

template <typename R>
lsw_status fgmres_run(const lsw_green* g, const double* chi, const lsw_hmatrix* h, const typename Cx<R>::T* b,
                      typename Cx<R>::T* x, int nb, int m, int max_iter, double tol, std::vector<SrcInfo>& info,
                      cudaStream_t st, Learned* lp = nullptr) {
    typedef typename Cx<R>::T C;
    typedef std::complex<double> Z;
    const long long n = (long long)g->nz * g->nx;
    m = std::max(1, std::min(m, 128));
    DevBuf V, Zb, vj, zj, w, hc, hc2, work, dn, act, ysc, yb;
    LSW_TRY(V.alloc(sizeof(C) * n * (m + 1) * nb, st));
    LSW_TRY(Zb.alloc(sizeof(C) * n * m * nb, st));
    LSW_TRY(vj.alloc(sizeof(C) * n * nb, st));
    LSW_TRY(zj.alloc(sizeof(C) * n * nb, st));
    LSW_TRY(w.alloc(sizeof(C) * n * nb, st));
    LSW_TRY(hc.alloc(sizeof(C) * (m + 1) * nb, st));
    LSW_TRY(hc2.alloc(sizeof(C) * (m + 1) * nb, st));
    LSW_TRY(ysc.alloc(sizeof(double) * nb, st));
    LSW_TRY(yb.alloc(sizeof(C) * m * nb, st));
    LSW_CUDA(cudaMemsetAsync(Zb.p, 0, sizeof(C) * n * m * nb, st));
    LSW_CUDA(cudaMemsetAsync(x, 0, sizeof(C) * n * nb, st));
    std::vector<double> nrmb, nr;
    LSW_TRY(host_norms<R>(b, n, nb, dn, nrmb, st));
    info.assign(nb, SrcInfo());
    std::vector<int> done(nb, 0);
    for (int s = 0; s < nb; ++s)
        if (!(nrmb[s] > 0)) { done[s] = 1; info[s].status = LSW_OK; info[s].rel = 0; }
    std::vector<Z> H((size_t)nb * (m + 1) * m), gv((size_t)nb * (m + 1)), cs((size_t)nb * m), sn((size_t)nb * m);
    std::vector<C> hh((size_t)(m + 1) * nb), hh2((size_t)(m + 1) * nb), yh((size_t)m * nb);
    std::vector<int> kused(nb, 0), conv(nb, 0), its(nb, 0);
    std::vector<double> scale(nb), wstart(nb);
    const C one_ = mk((R)1, (R)0), zero_ = mk((R)0, (R)0), mone = mk((R)-1, (R)0);
    int total = 0;
    const size_t pitchV = sizeof(C) * n * (m + 1), pitchZ = sizeof(C) * n * m, row = sizeof(C) * n;
    StepGraph sg;
    while (true) {
        // r = b - A x  (RESIDUAL gives x - G0V x - b = -r)
        LSW_TRY(op_full<R>(g, chi, LSW_OP_RESIDUAL, x, b, w.as<C>(), nb, work, st));
        LSW_TRY(host_norms<R>(w.as<C>(), n, nb, dn, nr, st));
        int left = 0;
        for (int s = 0; s < nb; ++s) {
            if (done[s]) continue;
            const double rel = std::sqrt(nr[s] / nrmb[s]);
            info[s].rel = rel;
            info[s].iters = its[s];
            if (!std::isfinite(rel)) { done[s] = 1; info[s].status = LSW_ERR_NUMERIC; continue; }
            if (rel <= tol) { done[s] = 1; info[s].status = LSW_OK; continue; }
            if (total >= max_iter) { done[s] = 1; info[s].status = LSW_ERR_NOT_CONVERGED; continue; }
            ++left;
        }
        if (!left) break;
        for (int s = 0; s < nb; ++s) {
            const double beta = std::sqrt(nr[s]);
            wstart[s] = beta;
            scale[s] = (!done[s] && beta > 0) ? -1.0 / beta : 0.0;
            for (int i = 0; i <= m; ++i) gv[(size_t)s * (m + 1) + i] = 0;
            gv[(size_t)s * (m + 1)] = done[s] ? 0.0 : beta;
            kused[s] = 0;
            conv[s] = done[s];
        }
        LSW_TRY(up(ysc, scale, st));
        k_scale_cast<C, C><<<gridn(n * nb), 256, 0, st>>>(w.as<C>(), vj.as<C>(), ysc.as<double>(), n, nb);
        LSW_LAUNCH_CHECK();
        LSW_CUDA(cudaMemcpy2DAsync(V.p, pitchV, vj.p, row, row, nb, cudaMemcpyDeviceToDevice, st));
        const bool learned = lp && lp->fno && !lp->off;
        bool stalled = false;
        int j = 0;
        for (; j < m; ++j) {
            // z_j = H v_j (or the network's z_j) ; w = A z_j
            if (learned) {
                LSW_TRY(fno_apply_precond(lp->fno, g, chi, vj.p, zj.p, nb, sizeof(R) == 8 ? LSW_C128 : LSW_C64, st));
                LSW_TRY(op_full<R>(g, chi, LSW_OP_RESIDUAL, zj.as<C>(), nullptr, w.as<C>(), nb, work, st));
            } else {
                LSW_TRY(sg.run(st, [&](cudaStream_t ss) -> lsw_status {
                    if (h) LSW_TRY(apply_h<R>(h, vj.as<C>(), zj.as<C>(), nb, ss));
                    else LSW_CUDA(cudaMemcpyAsync(zj.p, vj.p, sizeof(C) * n * nb, cudaMemcpyDeviceToDevice, ss));
                    return op_full<R>(g, chi, LSW_OP_RESIDUAL, zj.as<C>(), nullptr, w.as<C>(), nb, work, ss);
                }));
            }
            LSW_CUDA(cudaMemcpy2DAsync(Zb.as<char>() + row * j, pitchZ, zj.p, row, row, nb, cudaMemcpyDeviceToDevice, st));
            // two passes of classical Gram-Schmidt against v_0..v_j, then the
            // norm of what is left: the coefficients of both passes and the
            // norms come back to the host together, one wait per iteration
            std::vector<Z> hsum((size_t)nb * (j + 1), 0.0);
            // per pass the basis is read twice and w three times
            KTimer kt_gs("arnoldi_gs", st, sizeof(C) * (double)n * nb * (4.0 * (j + 1) + 7.0), 0.0);
            for (int pass = 0; pass < 2; ++pass) {
                C* hcp = pass == 0 ? hc.as<C>() : hc2.as<C>();
                LSW_TRY(gemm<R>('C', 'N', j + 1, 1, (int)n, one_, V.as<C>(), (int)n, n * (m + 1), w.as<C>(), (int)n, n,
                                zero_, hcp, m + 1, m + 1, nb, st));
                LSW_TRY(gemm<R>('N', 'N', (int)n, 1, j + 1, mone, V.as<C>(), (int)n, n * (m + 1), hcp, m + 1, m + 1,
                                one_, w.as<C>(), (int)n, n, nb, st));
            }
            if (!dn.p) LSW_TRY(dn.alloc(sizeof(double) * nb, st));
            LSW_TRY(norms2<R>(w.as<C>(), n, nb, dn.as<double>(), st));
            nr.resize(nb);
            LSW_CUDA(cudaMemcpyAsync(hh.data(), hc.p, sizeof(C) * (m + 1) * nb, cudaMemcpyDeviceToHost, st));
            LSW_CUDA(cudaMemcpyAsync(hh2.data(), hc2.p, sizeof(C) * (m + 1) * nb, cudaMemcpyDeviceToHost, st));
            LSW_CUDA(cudaMemcpyAsync(nr.data(), dn.p, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
            LSW_CUDA(cudaStreamSynchronize(st));
            for (int s = 0; s < nb; ++s)
                for (int i = 0; i <= j; ++i) {
                    const C v = hh[(size_t)s * (m + 1) + i], v2 = hh2[(size_t)s * (m + 1) + i];
                    hsum[(size_t)s * (j + 1) + i] += Z((double)v.x + (double)v2.x, (double)v.y + (double)v2.y);
                }
            for (int s = 0; s < nb; ++s) scale[s] = (!conv[s] && nr[s] > 0) ? 1.0 / std::sqrt(nr[s]) : 0.0;
            LSW_TRY(up(ysc, scale, st));
            k_scale_cast<C, C><<<gridn(n * nb), 256, 0, st>>>(w.as<C>(), vj.as<C>(), ysc.as<double>(), n, nb);
            LSW_LAUNCH_CHECK();
            LSW_CUDA(cudaMemcpy2DAsync(V.as<char>() + row * (j + 1), pitchV, vj.p, row, row, nb,
                                       cudaMemcpyDeviceToDevice, st));
            ++total;
            int still = 0;
            for (int s = 0; s < nb; ++s) {
                if (conv[s]) continue;
                Z* Hs = &H[(size_t)s * (m + 1) * m];     // column-major (m+1) x m
                for (int i = 0; i <= j; ++i) Hs[(size_t)j * (m + 1) + i] = hsum[(size_t)s * (j + 1) + i];
                Hs[(size_t)j * (m + 1) + j + 1] = std::sqrt(nr[s]);
                Z* cS = &cs[(size_t)s * m];
                Z* sS = &sn[(size_t)s * m];
                for (int i = 0; i < j; ++i) {       // earlier rotations
                    const Z a = Hs[(size_t)j * (m + 1) + i], bq = Hs[(size_t)j * (m + 1) + i + 1];
                    Hs[(size_t)j * (m + 1) + i] = std::conj(cS[i]) * a + std::conj(sS[i]) * bq;
                    Hs[(size_t)j * (m + 1) + i + 1] = -sS[i] * a + cS[i] * bq;
                }
                const Z a = Hs[(size_t)j * (m + 1) + j], bq = Hs[(size_t)j * (m + 1) + j + 1];
                const double den = std::sqrt(std::norm(a) + std::norm(bq));
                // a direction that adds nothing (den == 0) leaves the residual
                // estimate where it was
                Z c_ = 0.0, s_ = 1.0;
                if (den > 0) { c_ = a / den; s_ = bq / den; }
                cS[j] = c_;
                sS[j] = s_;
                Hs[(size_t)j * (m + 1) + j] = std::conj(c_) * a + std::conj(s_) * bq;
                Hs[(size_t)j * (m + 1) + j + 1] = 0;
                Z* gs = &gv[(size_t)s * (m + 1)];
                const Z g0 = gs[j];
                gs[j] = std::conj(c_) * g0;
                gs[j + 1] = -s_ * g0;
                kused[s] = j + 1;
                ++its[s];
                const double est = std::abs(gs[j + 1]) / std::sqrt(nrmb[s]);
                if (est <= tol || nr[s] == 0) conv[s] = 1;
                else ++still;
                if (learned && (j + 1) % kProbe == 0) {
                    if (std::abs(gs[j + 1]) > kProbeRatio * wstart[s]) stalled = true;
                    wstart[s] = std::abs(gs[j + 1]);
                }
            }
            if (stalled) lp->off = true;
            if (!still || total >= max_iter || stalled) { ++j; break; }
        }
        // a stalled cycle's directions came from a network that does not
        // help here: its update is dropped and the next cycle restarts from x
        if (stalled && j <= kProbe) continue;
        // x += Z y  with R y = g (back substitution per source)
        for (int s = 0; s < nb; ++s) {
            for (int i = 0; i < m; ++i) yh[(size_t)s * m + i] = mk((R)0, (R)0);
            if (done[s]) continue;
            const int k = kused[s];
            const Z* Hs = &H[(size_t)s * (m + 1) * m];
            const Z* gs = &gv[(size_t)s * (m + 1)];
            std::vector<Z> y(k);
            double dmax = 0;
            for (int i = 0; i < k; ++i) dmax = std::max(dmax, std::abs(Hs[(size_t)i * (m + 1) + i]));
            const double dmin = learned ? 1e-6 * dmax : 0.0;
            for (int i = k - 1; i >= 0; --i) {
                Z acc = gs[i];
                for (int q = i + 1; q < k; ++q) acc -= Hs[(size_t)q * (m + 1) + i] * y[q];
                const Z d = Hs[(size_t)i * (m + 1) + i];
                y[i] = std::abs(d) > dmin ? acc / d : Z(0);
                yh[(size_t)s * m + i] = mk((R)y[i].real(), (R)y[i].imag());
            }
        }
        LSW_CUDA(cudaMemcpyAsync(yb.p, yh.data(), sizeof(C) * m * nb, cudaMemcpyHostToDevice, st));
        // only the j columns of Z written in this cycle take part
        LSW_TRY(gemm<R>('N', 'N', (int)n, 1, j, one_, Zb.as<C>(), (int)n, n * m, yb.as<C>(), m, m, one_, x, (int)n, n, nb,
                        st));
    }
    return LSW_OK;
}

template <typename R>
lsw_status inner_run(int method, const lsw_green* g, const double* chi, const lsw_hmatrix* h,
                     const typename Cx<R>::T* b, typename Cx<R>::T* x, int nb, const lsw_solve_params* sp, double tol,
                     std::vector<SrcInfo>& info, cudaStream_t st, Learned* lp) {
    if (method == LSW_FGMRES) return fgmres_run<R>(g, chi, h, b, x, nb, sp->restart, sp->max_iter, tol, info, st, lp);
    return series_run<R>(g, chi, h, b, x, nb, sp->max_iter, tol, info, st);
}

// Final FP64 relative residual of a field held in precision R.
template <typename R>
lsw_status fp64_residual(const lsw_green* g, const double* chi, const typename Cx<R>::T* u,
                         const typename Cx<R>::T* u0, int nb, std::vector<double>& rel, cudaStream_t st) {
    typedef typename Cx<R>::T C;
    const long long n = (long long)g->nz * g->nx;
    DevBuf u64, b64, a, work, dn;
    const double2* pu = reinterpret_cast<const double2*>(u);
    const double2* pb = reinterpret_cast<const double2*>(u0);
    if (sizeof(R) != 8) {
        LSW_TRY(u64.alloc(sizeof(double2) * n * nb, st));
        LSW_TRY(b64.alloc(sizeof(double2) * n * nb, st));
        k_scale_cast<C, double2><<<gridn(n * nb), 256, 0, st>>>(u, u64.as<double2>(), nullptr, n, nb);
        LSW_LAUNCH_CHECK();
        k_scale_cast<C, double2><<<gridn(n * nb), 256, 0, st>>>(u0, b64.as<double2>(), nullptr, n, nb);
        LSW_LAUNCH_CHECK();
        pu = u64.as<double2>();
        pb = b64.as<double2>();
    }
    LSW_TRY(a.alloc(sizeof(double2) * n * nb, st));
    LSW_TRY(op_full<double>(g, chi, LSW_OP_RESIDUAL, pu, pb, a.as<double2>(), nb, work, st));
    std::vector<double> na, n0;
    LSW_TRY(host_norms<double>(a.as<double2>(), n, nb, dn, na, st));
    DevBuf dn2;
    LSW_TRY(host_norms<double>(pb, n, nb, dn2, n0, st));
    rel.resize(nb);
    for (int s = 0; s < nb; ++s) rel[s] = n0[s] > 0 ? std::sqrt(na[s] / n0[s]) : 0.0;
    return LSW_OK;
}

// Mixed precision: FP64 residual outside, FP32 corrections inside.
lsw_status mixed_run(const lsw_green* g, const double* chi, const lsw_hmatrix* h, const double2* u0, double2* u,
                     int nb, const lsw_solve_params* sp, std::vector<SrcInfo>& info, std::vector<int>& outer,
                     cudaStream_t st, Learned* lp) {
    const long long n = (long long)g->nz * g->nx;
    DevBuf a, r32, d32, work, dn, act, sc;
    LSW_TRY(a.alloc(sizeof(double2) * n * nb, st));
    LSW_TRY(r32.alloc(sizeof(float2) * n * nb, st));
    LSW_TRY(d32.alloc(sizeof(float2) * n * nb, st));
    LSW_CUDA(cudaMemsetAsync(u, 0, sizeof(double2) * n * nb, st));
    std::vector<double> n0, na;
    LSW_TRY(host_norms<double>(u0, n, nb, dn, n0, st));
    info.assign(nb, SrcInfo());
    outer.assign(nb, 0);
    std::vector<int> active(nb, 1);
    std::vector<double> scale(nb);
    for (int k = 0;; ++k) {
        LSW_TRY(op_full<double>(g, chi, LSW_OP_RESIDUAL, u, u0, a.as<double2>(), nb, work, st));
        LSW_TRY(host_norms<double>(a.as<double2>(), n, nb, dn, na, st));
        int left = 0;
        for (int s = 0; s < nb; ++s) {
            if (!active[s]) continue;
            const double rel = n0[s] > 0 ? std::sqrt(na[s] / n0[s]) : 0.0;
            info[s].rel = rel;
            outer[s] = k;
            if (!std::isfinite(rel)) { info[s].status = LSW_ERR_NUMERIC; active[s] = 0; continue; }
            if (rel <= sp->tol) { info[s].status = LSW_OK; active[s] = 0; continue; }
            if (k == sp->max_outer) { info[s].status = LSW_ERR_NOT_CONVERGED; active[s] = 0; continue; }
            ++left;
        }
        if (!left) break;
        // r = psi0 - (I - G0V) psi = -a, cast to FP32 (zero for finished sources)
        for (int s = 0; s < nb; ++s) scale[s] = active[s] ? -1.0 : 0.0;
        LSW_TRY(up(sc, scale, st));
        k_scale_cast<double2, float2><<<gridn(n * nb), 256, 0, st>>>(a.as<double2>(), r32.as<float2>(), sc.as<double>(),
                                                                       n, nb);
        LSW_LAUNCH_CHECK();
        std::vector<SrcInfo> in;
        LSW_TRY(inner_run<float>(sp->method, g, chi, h, r32.as<float2>(), d32.as<float2>(), nb, sp, sp->inner_tol, in,
                                 st, lp));
        for (int s = 0; s < nb; ++s)
            if (active[s]) info[s].iters += in[s].iters;
        LSW_TRY(up(act, active, st));
        k_add_up<float2><<<gridn(n * nb), 256, 0, st>>>(u, d32.as<float2>(), act.as<int>(), n, nb);
        LSW_LAUNCH_CHECK();
    }
    return LSW_OK;
}

}  // namespace

lsw_status solve(const lsw_green* g, const double* chi, const lsw_hmatrix* h, const void* u0, void* u, int nb,
                 const lsw_solve_params* sp, lsw_solve_info* out, cudaStream_t st, Learned* lp) {
    std::vector<SrcInfo> info;
    std::vector<int> outer(nb, 0);
    std::vector<double> rel;
    const int method = sp->method;
    if (sp->prec == LSW_MIXED) {
        LSW_TRY(mixed_run(g, chi, h, (const double2*)u0, (double2*)u, nb, sp, info, outer, st, lp));
        for (int s = 0; s < nb; ++s) rel.push_back(info[s].rel);
    } else if (sp->prec == LSW_C128) {
        LSW_TRY(inner_run<double>(method, g, chi, h, (const double2*)u0, (double2*)u, nb, sp, sp->tol, info, st, lp));
        LSW_TRY(fp64_residual<double>(g, chi, (const double2*)u, (const double2*)u0, nb, rel, st));
    } else {
        LSW_TRY(inner_run<float>(method, g, chi, h, (const float2*)u0, (float2*)u, nb, sp, sp->tol, info, st, lp));
        LSW_TRY(fp64_residual<float>(g, chi, (const float2*)u, (const float2*)u0, nb, rel, st));
    }
    lsw_status first = LSW_OK;
    for (int s = 0; s < nb; ++s) {
        out[s].iterations = info[s].iters;
        out[s].outer = outer[s];
        out[s].status = info[s].status;
        out[s].fallback = lp && lp->off ? 1 : 0;
        out[s].rel_residual = rel[s];
        if (first == LSW_OK && info[s].status != LSW_OK) first = info[s].status;
    }
    return first;
}

}  // namespace lsw

using namespace lsw;

namespace {
lsw_status check_solve(const lsw_green* g, const double* chi, const lsw_hmatrix* h, const void* u0, void* u,
                       int nbatch, const lsw_solve_params* sp, lsw_solve_info* info) {
    if (!g || !chi || !sp || !info || nbatch < 0) return LSW_ERR_INVALID_ARG;
    if (nbatch == 0) return LSW_OK;
    if (!u0 || !u || u0 == u) return LSW_ERR_INVALID_ARG;
    if (sp->prec != LSW_C128 && sp->prec != LSW_C64 && sp->prec != LSW_MIXED) return LSW_ERR_INVALID_ARG;
    if (sp->method != LSW_SERIES && sp->method != LSW_FGMRES) return LSW_ERR_INVALID_ARG;
    if (sp->max_iter < 0 || !(sp->tol > 0) || (sp->method == LSW_FGMRES && sp->restart < 1)) return LSW_ERR_INVALID_ARG;
    if (sp->prec == LSW_MIXED && (!(sp->inner_tol > 0) || sp->max_outer < 0)) return LSW_ERR_INVALID_ARG;
    if (h) {
        const int hp = hmatrix_prec(h);
        const int want = sp->prec == LSW_C128 ? LSW_C128 : LSW_C64;
        if (hp != want) return LSW_ERR_INVALID_ARG;
    }
    return LSW_OK;
}
}  // namespace

extern "C" lsw_status lsw_solve_series(const lsw_green* g, const double* chi, const lsw_hmatrix* h, const void* u0,
                                       void* u, int nbatch, const lsw_solve_params* sp, lsw_solve_info* info,
                                       void* stream) {
    LSW_TRY(check_solve(g, chi, h, u0, u, nbatch, sp, info));
    if (nbatch == 0) return LSW_OK;
    return solve(g, chi, h, u0, u, nbatch, sp, info, reinterpret_cast<cudaStream_t>(stream), nullptr);
}

extern "C" lsw_status lsw_solve_learned(const lsw_green* g, const double* chi, const lsw_fno* fno,
                                        const lsw_hmatrix* h, const void* u0, void* u, int nbatch,
                                        const lsw_solve_params* sp, lsw_solve_info* info, void* stream) {
    if (!fno) return LSW_ERR_INVALID_ARG;
    LSW_TRY(check_solve(g, chi, h, u0, u, nbatch, sp, info));
    if (sp->method != LSW_FGMRES) return LSW_ERR_INVALID_ARG;
    if (nbatch == 0) return LSW_OK;
    if (!fno_matches(fno, g)) return LSW_ERR_INVALID_ARG;
    Learned lp;
    lp.fno = fno;
    return solve(g, chi, h, u0, u, nbatch, sp, info, reinterpret_cast<cudaStream_t>(stream), &lp);
}
