// Preconditioners H ~ (I - G0 V)^-1 (Sec. 2.3-2.4): randomized sketches of
// blocks of G0 V (Algorithm 2), the simple low-rank + Sherman-Morrison-
// Woodbury preconditioner (Eq. 12), and the randomized HODLR approximation
// of I - G0 V with its recursive block inversion (Sec. 2.4, Fig. 1).
//
// HODLR storage on the device.  Node (l, c) is node c of level l; every node
// of a level has n_l = n / 2^l unknowns (power-of-two grids, halving splits),
// numbered in tree order: leaves left to right, cells of a leaf in strip
// order.  Block (l, c) -- rows node c, columns its sibling c^1 -- is
// U_l[c] W_l[c]^H with U_l, W_l arrays of 2^l column-major n_l x r factors;
// the 2^L dense leaves are D[c], n_L x n_L.  The blocks inside node (l, c)
// are therefore contiguous ranges of every deeper level's arrays, which turns
// each operation on a subtree into a few strided batched products.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <initializer_list>
#include <atomic>
#include <cmath>
#include <map>
#include <memory>
#include <new>
#include <type_traits>
#include <vector>

#include "lsw_internal.cuh"

namespace lsw {

// ------------------------------------------------------------- cluster tree
struct Tree {
    int nz = 0, nx = 0, L = 0, split = 0, n = 0;
    std::vector<int4> box;           // node (l, c) at (1 << l) - 1 + c: (z0, z1, x0, x1)
    std::vector<int> perm;           // tree index -> grid index
    int nl(int l) const { return n >> l; }
    int4 node(int l, int c) const { return box[(1 << l) - 1 + c]; }

    lsw_status init(int nz_, int nx_, int levels, int split_) {
        nz = nz_; nx = nx_; L = levels; split = split_; n = nz * nx;
        box.assign((size_t)(2 << L) - 1, make_int4(0, 0, 0, 0));
        box[0] = make_int4(0, nz, 0, nx);
        for (int l = 0; l < L; ++l)
            for (int c = 0; c < (1 << l); ++c) {
                const int4 b = node(l, c);
                const int ez = b.y - b.x, ex = b.w - b.z;
                const bool along_x = split == LSW_SPLIT_STRIPS || ex >= ez;
                int4 a = b, d = b;
                if (along_x) {
                    if (ex < 2) return LSW_ERR_INVALID_ARG;
                    const int xm = b.z + ex / 2;
                    a.w = xm; d.z = xm;
                } else {
                    if (ez < 2) return LSW_ERR_INVALID_ARG;
                    const int zm = b.x + ez / 2;
                    a.y = zm; d.x = zm;
                }
                box[(2 << l) - 1 + 2 * c] = a;
                box[(2 << l) - 1 + 2 * c + 1] = d;
            }
        perm.clear();
        perm.reserve(n);
        for (int c = 0; c < (1 << L); ++c) {
            const int4 b = node(L, c);
            for (int ix = b.z; ix < b.w; ++ix)
                for (int iz = b.x; iz < b.y; ++iz) perm.push_back(ix * nz + iz);
        }
        return LSW_OK;
    }

    // position, inside the box of node (l-1, 0), of the unknowns of its child
    // `which` (tree order); the same for every parent of the level.
    std::vector<int> child_map(int l, int which) const {
        const int4 P = node(l - 1, 0);
        const int pz = P.y - P.x;
        const int m = nl(l), off = which * m;   // child's first tree index inside parent 0
        std::vector<int> out(m);
        for (int i = 0; i < m; ++i) {
            const int g = perm[off + i];
            const int ix = g / nz, iz = g % nz;
            out[i] = (ix - P.z) * pz + (iz - P.x);
        }
        return out;
    }
};

// Large H-matrix arrays come from the device's stream-ordered pool (which
// keeps freed memory mapped: the next build of the same size reuses it
// without new mappings).  The allocation is complete before the call
// returns; a release first waits for the device, as cudaFree would.
inline lsw_status pool_alloc(void** p, size_t bytes) {
    if (cudaMallocAsync(p, bytes, 0) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return LSW_ERR_OOM;
    }
    if (cudaStreamSynchronize(0) != cudaSuccess) return LSW_ERR_CUDA;
    return LSW_OK;
}
inline void pool_free_all(std::initializer_list<const std::vector<void*>*> lists) {
    cudaDeviceSynchronize();
    for (auto v : lists)
        for (void* p : *v)
            if (p) cudaFreeAsync(p, 0);
}

template <typename R> struct HStore {
    typedef typename Cx<R>::T C;
    int L = 0, r = 0, n = 0;
    C* D = nullptr;
    std::vector<C*> U, W;   // index by level, [0] unused
    size_t bytes = 0;
    int nl(int l) const { return n >> l; }
    lsw_status alloc(int L_, int r_, int n_) {
        L = L_; r = r_; n = n_;
        const int nL = nl(L);
        const size_t dbytes = sizeof(C) * (size_t)n * nL;
        LSW_TRY(pool_alloc(reinterpret_cast<void**>(&D), dbytes));
        bytes = dbytes;
        U.assign(L + 1, nullptr);
        W.assign(L + 1, nullptr);
        for (int l = 1; l <= L; ++l) {
            const size_t b = sizeof(C) * (size_t)n * r;   // 2^l blocks x n_l x r
            LSW_TRY(pool_alloc(reinterpret_cast<void**>(&U[l]), b));
            LSW_TRY(pool_alloc(reinterpret_cast<void**>(&W[l]), b));
            bytes += 2 * b;
        }
        return LSW_OK;
    }
    void release() {
        if (!D && U.empty() && W.empty()) return;
        std::vector<void*> a{D}, u(U.begin(), U.end()), w(W.begin(), W.end());
        pool_free_all({&a, &u, &w});
        D = nullptr;
        U.clear();
        W.clear();
    }
};

// The dense leaves of the matrix being inverted hold their inverses: the
// original leaves are inverted up front, in batches on another stream
// (leaves [end[b-1], end[b]) are ready once ready[b] has fired), and every
// rank-r update D += U V^H that a Schur complement S = D - C A^-1 B brings
// to a leaf is folded into its inverse at once by Woodbury.
template <typename R> struct LeafUpd {
    std::vector<cudaEvent_t> ready;
    std::vector<int> end;
    // level l's off-diagonal blocks of the matrix being inverted are
    // sketched once level_done[l] has fired (none: already complete)
    std::vector<cudaEvent_t> level_done;
    lsw_status wait_level(int l, cudaStream_t st) const {
        if (l >= 0 && l < (int)level_done.size() && level_done[l]) LSW_CUDA(cudaStreamWaitEvent(st, level_done[l], 0));
        return LSW_OK;
    }
    // make st wait until every leaf up to `last` has its inverse
    lsw_status wait(int last, cudaStream_t st) const {
        for (size_t b = 0; b < end.size(); ++b)
            if (last < end[b]) {
                LSW_CUDA(cudaStreamWaitEvent(st, ready[b], 0));
                break;
            }
        return LSW_OK;
    }
};

// H kept as BF16 pairs (re, im in one 32-bit word) after an FP32 build;
// only the whole-matrix product runs on this storage.
struct HStoreB {
    int L = 0, r = 0, n = 0;
    int rp = 0;                       // columns per block of the tiled levels
    uint32_t* D = nullptr;
    std::vector<uint32_t*> U, W;
    std::vector<int> ulay, wlay;      // FAC_* storage of each level's U and W
    size_t bytes = 0;
    int nl(int l) const { return n >> l; }
    void release() {
        if (!D && U.empty() && W.empty()) return;
        std::vector<void*> a{D}, u(U.begin(), U.end()), w(W.begin(), W.end());
        pool_free_all({&a, &u, &w});
        D = nullptr;
        U.clear();
        W.clear();
    }
};

}  // namespace lsw

struct lsw_hmatrix {
    int kind = 0, prec = 0, n = 0, r = 0, L = 0, nz = 0, nx = 0;
    lsw::Tree tree;
    int* perm_d = nullptr;
    lsw::HStore<float> h32;
    lsw::HStore<double> h64;
    lsw::HStoreB hb;         // BF16 storage (bf16 true): h32 is released
    bool bf16 = false;
    void* smwU = nullptr;    // n x r
    void* smwW = nullptr;    // n x r
    void* smwZ = nullptr;    // r x r
    size_t bytes = 0;
};

namespace lsw {

namespace {

int gridn(long long n, int bs = 256) {
    long long g = (n + bs - 1) / bs;
    return (int)std::max<long long>(1, std::min<long long>(g, 152LL * 32));
}

constexpr uint32_t TAG_BUILD = 1, TAG_GLOBAL = 2, TAG_RECOMPRESS = 3;

uint32_t stream_w2(uint32_t tag, uint32_t op, uint32_t lvl, uint32_t node) {
    return ((tag & 0xF) << 28) | ((op & 0xF) << 24) | ((lvl & 0xFF) << 16) | (node & 0xFFFF);
}

// ------------------------------------------------------------- kernels
// dst vector (b = (c >> 1) * 2rp + (c & 1) * rp + j) at map[which(c)][i]
//   <- src block c, column j, row i     (which(c) = (c ^ flip) & 1)
template <typename C>
__global__ void k_scatter_blocks(const C* __restrict__ src, int nb, int rp, int nblk, const int* __restrict__ map,
                                 int flip, long long boxn, C* __restrict__ dst) {
    const long long tot = (long long)nblk * rp * nb;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e / ((long long)rp * nb));
        const long long r = e - (long long)c * rp * nb;
        const int j = (int)(r / nb), i = (int)(r - (long long)j * nb);
        const int which = (c ^ flip) & 1;
        const long long b = (long long)(c >> 1) * 2 * rp + (c & 1) * rp + j;
        dst[b * boxn + map[which * nb + i]] = src[e];
    }
}

template <typename C>
__global__ void k_gather_blocks(const C* __restrict__ src, int nb, int rp, int nblk, const int* __restrict__ map,
                                int flip, long long boxn, C* __restrict__ dst) {
    const long long tot = (long long)nblk * rp * nb;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e / ((long long)rp * nb));
        const long long r = e - (long long)c * rp * nb;
        const int j = (int)(r / nb), i = (int)(r - (long long)j * nb);
        const int which = (c ^ flip) & 1;
        const long long b = (long long)(c >> 1) * 2 * rp + (c & 1) * rp + j;
        dst[e] = src[b * boxn + map[which * nb + i]];
    }
}

// generic map scatter / gather for one block of k columns
template <typename C>
__global__ void k_scatter_map(const C* __restrict__ src, int m, int k, const int* __restrict__ map, long long boxn,
                              C* __restrict__ dst) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)m * k; e += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(e / m), i = (int)(e - (long long)j * m);
        dst[j * boxn + map[i]] = src[e];
    }
}
template <typename C>
__global__ void k_gather_map(const C* __restrict__ src, int m, int k, const int* __restrict__ map, long long boxn,
                             C* __restrict__ dst) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)m * k; e += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(e / m), i = (int)(e - (long long)j * m);
        dst[e] = src[j * boxn + map[i]];
    }
}

// x_tree[s][i] = x_grid[s][perm[i]]   (dir = 0)   or the inverse (dir = 1)
template <typename C>
__global__ void k_permute(const C* __restrict__ src, C* __restrict__ dst, const int* __restrict__ perm, int n, int nb,
                          int dir) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * nb; e += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(e / n), i = (int)(e - (long long)s * n);
        const long long g = (long long)s * n + perm[i];
        if (dir == 0) dst[e] = src[g];
        else dst[g] = src[e];
    }
}

// Dense leaf of I - Gt diag(chi): entry (i, j) of leaf c, tree order.
template <typename C>
__global__ void k_leaf_assemble(const double2* __restrict__ table, int nz, const double* __restrict__ chi,
                                const int* __restrict__ perm, int nL, int nleaf, C* __restrict__ D) {
    const long long per = (long long)nL * nL;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < per * nleaf; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e / per);
        const long long r = e - (long long)c * per;
        const int j = (int)(r / nL), i = (int)(r - (long long)j * nL);
        const int gi = perm[c * nL + i], gj = perm[c * nL + j];
        const int dz = abs(gi % nz - gj % nz), dx = abs(gi / nz - gj / nz);
        const double2 g = table[dx * (nz + 1) + dz];
        const double ch = chi[gj];
        C v;
        v.x = (i == j ? 1.0 : 0.0) - g.x * ch;
        v.y = -g.y * ch;
        D[e] = v;
    }
}

// Uc_b = [U_b | X rows of block b],  Wc_b = [W_b | Y rows of block b ^ 1]
template <typename C>
__global__ void k_concat(const C* __restrict__ U, const C* __restrict__ W, const C* __restrict__ X, const C* __restrict__ Y,
                         int nb, int r, int ldx, int nblk, C* __restrict__ Uc, C* __restrict__ Wc) {
    const long long per = (long long)nb * 2 * r;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < per * nblk; e += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(e / per);
        const long long q = e - (long long)b * per;
        const int col = (int)(q / nb), i = (int)(q - (long long)col * nb);
        if (col < r) {
            Uc[e] = U[(long long)b * nb * r + (long long)col * nb + i];
            Wc[e] = W[(long long)b * nb * r + (long long)col * nb + i];
        } else {
            const int cc = col - r;
            Uc[e] = X[(long long)cc * ldx + (long long)b * nb + i];
            Wc[e] = Y[(long long)cc * ldx + (long long)(b ^ 1) * nb + i];
        }
    }
}

// M_b += I for a batch of r x r matrices (stride r * r).
template <typename C>
__global__ void k_eye_plus(C* M, int r, int batch) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < r * batch; e += gridDim.x * blockDim.x) {
        const int b = e / r, i = e - b * r;
        M[(long long)b * r * r + (long long)i * r + i].x += 1;
    }
}

template <typename C>
__global__ void k_eye_minus(C* M, int r) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < r * r; e += gridDim.x * blockDim.x) {
        const int j = e / r, i = e - j * r;
        C v = M[e];
        v.x = (i == j ? 1 : 0) - v.x;
        v.y = -v.y;
        M[e] = v;
    }
}

template <typename C>
__global__ void k_copy(const C* __restrict__ s, C* __restrict__ d, long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) d[e] = s[e];
}

template <typename C, typename R>
__global__ void k_scale_copy(const C* __restrict__ s, C* __restrict__ d, long long n, R a) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        C v = s[e];
        v.x *= a;
        v.y *= a;
        d[e] = v;
    }
}

template <typename C> C one() { C v; v.x = 1; v.y = 0; return v; }
template <typename C> C minus_one() { C v; v.x = -1; v.y = 0; return v; }
template <typename C> C zero() { C v; v.x = 0; v.y = 0; return v; }

template <typename T>
lsw_status upload(DevBuf& b, const std::vector<T>& v, cudaStream_t st) {
    LSW_TRY(b.alloc(sizeof(T) * std::max<size_t>(1, v.size()), st));
    if (!v.empty()) LSW_CUDA(cudaMemcpyAsync(b.p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st));
    return LSW_OK;
}

}  // namespace

// ------------------------------------------------------------- truncation
// Best rank-r part of Q Yt^H for a batch of blocks (Q: nb x rp, Yt: mb x rp):
// with Yt^H Yt = V diag(lam) V^H (FP64 Gram, FP64 eigen-decomposition), keep
// the r leading eigenvectors Vr:  U = alphaU Q Vr,  W = Yt Vr,  so
// U W^H = alphaU Q Vr Vr^H Yt^H.
template <typename R>
lsw_status truncate(const typename Cx<R>::T* Q, int nb, const typename Cx<R>::T* Yt, int mb, int rp, int r, int nblk,
                    typename Cx<R>::T alphaU, typename Cx<R>::T* Uout, long long sU, typename Cx<R>::T* Wout,
                    long long sW, cudaStream_t st) {
    typedef typename Cx<R>::T C;
    DevBuf G, V;
    LSW_TRY(G.alloc(sizeof(double2) * (size_t)nblk * rp * rp, st));
    LSW_TRY(V.alloc(sizeof(C) * (size_t)nblk * rp * rp, st));
    LSW_TRY(gram64<R>(Yt, mb, rp, (long long)mb * rp, nblk, G.as<double2>(), st));
    if (sizeof(R) == 4) LSW_TRY(heev_c64(G.as<double2>(), reinterpret_cast<float2*>(V.p), rp, nblk, st));
    else LSW_TRY(heev_jacobi<R>(G.as<double2>(), V.as<C>(), rp, nblk, st));
    const int rr = std::min(r, rp);
    if (rr < r) {
        LSW_CUDA(cudaMemsetAsync(Uout, 0, sizeof(C) * (size_t)sU * nblk, st));
        LSW_CUDA(cudaMemsetAsync(Wout, 0, sizeof(C) * (size_t)sW * nblk, st));
    }
    LSW_TRY(gemm<R>('N', 'N', nb, rr, rp, alphaU, Q, nb, (long long)nb * rp, V.as<C>(), rp, (long long)rp * rp,
                    zero<C>(), Uout, nb, sU, nblk, st));
    LSW_TRY(gemm<R>('N', 'N', mb, rr, rp, one<C>(), Yt, mb, (long long)mb * rp, V.as<C>(), rp, (long long)rp * rp,
                    zero<C>(), Wout, mb, sW, nblk, st));
    return LSW_OK;
}

// Thin QR of the sketch blocks (Algorithm 1, step 3): FP64 Householder for
// complex128; shifted Cholesky QR with FP64 Grams and factors for complex64.
template <typename R>
lsw_status qr_sketch(typename Cx<R>::T* A, int m, int k, long long sA, int batch, cudaStream_t st);
template <>
lsw_status qr_sketch<double>(double2* A, int m, int k, long long sA, int batch, cudaStream_t st) {
    return qr_explicit<double>(A, m, k, sA, batch, nullptr, st);
}
template <>
lsw_status qr_sketch<float>(float2* A, int m, int k, long long sA, int batch, cudaStream_t st) {
    return qr_sketch_c64(A, m, k, sA, batch, st);
}

// ---------------------------------------------------------------- sketches
// Randomized range finder (Algorithm 1/2) for nblk blocks of G0 V on boxes
// of one shape.  fwd(Xin, Yout): Yout = (G0 V)[s, t] Xin for every block;
// adj(Xin, Yout): Yout = (G0 V)[s, t]^H Xin.  Q receives the basis
// (ns x rp per block), Yt the projection (nt x rp).
template <typename R, typename F, typename A>
lsw_status range_finder(int ns, int nt, int rp, int q, int nblk, typename Cx<R>::T* Omega, typename Cx<R>::T* Q,
                        typename Cx<R>::T* Yt, F fwd, A adj, cudaStream_t st) {
    LSW_TRY(fwd(Omega, Q));
    LSW_TRY(qr_sketch<R>(Q, ns, rp, (long long)ns * rp, nblk, st));
    for (int it = 0; it < q; ++it) {
        LSW_TRY(adj(Q, Yt));
        LSW_TRY(qr_sketch<R>(Yt, nt, rp, (long long)nt * rp, nblk, st));
        LSW_TRY(fwd(Yt, Q));
        LSW_TRY(qr_sketch<R>(Q, ns, rp, (long long)ns * rp, nblk, st));
    }
    return adj(Q, Yt);
}

// One level of the HODLR build: every block (l, c) of I - G0 V is
// -(G0 V)[node c, node c^1], sketched on the box of the parent node.
template <typename R>
lsw_status build_level(const lsw_green* g, const double* chi, const Tree& tr, int l, int r, int rp, int q,
                       uint64_t seed, HStore<R>& H, const Spectrum& sp, cudaStream_t st) {
    typedef typename Cx<R>::T C;
    const int nblk = 1 << l, npar = 1 << (l - 1), nb = tr.nl(l);
    const int4 P0 = tr.node(l - 1, 0);
    const int bz = P0.y - P0.x, bx = P0.w - P0.z;
    const long long boxn = (long long)bz * bx;

    std::vector<int> maps = tr.child_map(l, 0);
    std::vector<int> m1 = tr.child_map(l, 1);
    maps.insert(maps.end(), m1.begin(), m1.end());
    std::vector<int2> org(npar);
    for (int p = 0; p < npar; ++p) {
        const int4 b = tr.node(l - 1, p);
        org[p] = make_int2(b.x, b.z);
    }
    std::vector<uint32_t> w2(nblk, stream_w2(TAG_BUILD, 0, 0, 0)), w3(nblk);
    for (int c = 0; c < nblk; ++c) w3[c] = ((uint32_t)l << 16) | (uint32_t)c;
    DevBuf dmap, dorg, dw2, dw3, om, qb, yt, vin, vout, work;
    LSW_TRY(upload(dmap, maps, st));
    LSW_TRY(upload(dorg, org, st));
    LSW_TRY(upload(dw2, w2, st));
    LSW_TRY(upload(dw3, w3, st));
    const size_t blk = (size_t)nblk * nb * rp;
    const long long nvec = (long long)npar * 2 * rp;
    LSW_TRY(om.alloc(sizeof(C) * blk, st));
    LSW_TRY(qb.alloc(sizeof(C) * blk, st));
    LSW_TRY(yt.alloc(sizeof(C) * blk, st));
    LSW_TRY(vin.alloc(sizeof(C) * nvec * boxn, st));
    LSW_TRY(vout.alloc(sizeof(C) * nvec * boxn, st));
    LSW_TRY(work.alloc(sizeof(C) * nvec * boxn * 2, st));
    LSW_TRY(gaussian_fill<R>(om.as<C>(), nb, rp, (long long)nb * rp, nblk, seed, dw2.as<uint32_t>(),
                             dw3.as<uint32_t>(), st));
    OpGeom geo{bz, bx, chi, tr.nz, dorg.as<int2>(), 2 * rp};
    const int* map = dmap.as<int>();
    // forward: probes on t (= c ^ 1), outputs on s (= c)
    auto fwd = [&](const C* X, C* Y) -> lsw_status {
        LSW_CUDA(cudaMemsetAsync(vin.p, 0, sizeof(C) * nvec * boxn, st));
        k_scatter_blocks<C><<<gridn((long long)blk), 256, 0, st>>>(X, nb, rp, nblk, map, 1, boxn, vin.as<C>());
        LSW_LAUNCH_CHECK();
        LSW_TRY(op_apply<R>(g, sp, geo, LSW_OP_PLAIN, vin.as<C>(), nullptr, vout.as<C>(), (int)nvec, work.as<C>(), st));
        k_gather_blocks<C><<<gridn((long long)blk), 256, 0, st>>>(vout.as<C>(), nb, rp, nblk, map, 0, boxn, Y);
        LSW_LAUNCH_CHECK();
        return LSW_OK;
    };
    auto adj = [&](const C* X, C* Y) -> lsw_status {
        LSW_CUDA(cudaMemsetAsync(vin.p, 0, sizeof(C) * nvec * boxn, st));
        k_scatter_blocks<C><<<gridn((long long)blk), 256, 0, st>>>(X, nb, rp, nblk, map, 0, boxn, vin.as<C>());
        LSW_LAUNCH_CHECK();
        LSW_TRY(op_apply<R>(g, sp, geo, LSW_OP_ADJOINT, vin.as<C>(), nullptr, vout.as<C>(), (int)nvec, work.as<C>(), st));
        k_gather_blocks<C><<<gridn((long long)blk), 256, 0, st>>>(vout.as<C>(), nb, rp, nblk, map, 1, boxn, Y);
        LSW_LAUNCH_CHECK();
        return LSW_OK;
    };
    LSW_TRY((range_finder<R>(nb, nb, rp, q, nblk, om.as<C>(), qb.as<C>(), yt.as<C>(), fwd, adj, st)));
    LSW_TRY(truncate<R>(qb.as<C>(), nb, yt.as<C>(), nb, rp, r, nblk, minus_one<C>(), H.U[l], (long long)nb * r, H.W[l],
                        (long long)nb * r, st));
    return LSW_OK;
}

// ------------------------------------------------------- subtree products
// The off-diagonal part of a subtree product, every level at once.  Level q
// of node (l, c) has cnt_q blocks of nb_q rows; block j's factors F_j, G_j
// (nb_q x r, column-major) are consecutive, stride nb_q * r.  For every
// level and block:
//     T_j = F_j^H X[rows of block j, or of its sibling j ^ 1 if swapA]
//     Y[rows of block b] += G_b' T_b'  with b' = b (or b ^ 1 if swapC)
// (X, Y: m x k, ld m, m = the node's rows).  Three launches: partial T over
// row chunks of every level, the fixed-order reduction of the partials, and
// one pass over Y adding every level's G T.
// factor entries as stored (complex FP32 / FP64, or a BF16 pair in 32 bits)
__device__ __forceinline__ float2 ldfac(const float2* p) { return *p; }
__device__ __forceinline__ double2 ldfac(const double2* p) { return *p; }
__device__ __forceinline__ float2 ldfac(const uint32_t* p) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
}

// Partial T over one chunk of CH rows: out (r x k) = F_chunk^H X_chunk.
// Rows go through shared memory in tiles of 32, stored row-major so that a
// thread reads 2 x 2 complex at a time; thread (microtile, row group) keeps a
// 4 x 4 block of outputs over every G-th row of the tile, and the row groups
// are summed in shared memory at the end.
template <typename C, typename FT>
__global__ void __launch_bounds__(256)
k_lr_partial(LrLevels<C, FT> lv, int m, int r, int k, const C* __restrict__ X, int swapA, C* __restrict__ P) {
    constexpr int TR = 32;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int rs = (r + 3) & ~3, ks = (k + 3) & ~3;       // columns rounded up to 4
    const int fsd = rs + 1, xsd = ks + 1;                 // odd row strides: conflict-free transposing stores
    C* Fs = reinterpret_cast<C*>(sm_raw);                 // TR x fsd
    C* Xs = Fs + TR * fsd;                                // TR x xsd
    C* Red = Xs + TR * xsd;                               // G x r x k
    int q = 0;
    while (q + 1 < lv.nlev && (int)blockIdx.x >= lv.chunk0[q + 1]) ++q;
    const int chn = blockIdx.x - lv.chunk0[q];
    const int CH = lv.ch[q], nb = lv.nb[q];
    const int row0 = chn * CH;
    const int j = row0 / nb, o = row0 - j * nb;
    const int src = swapA ? (j ^ 1) : j;
    const int flay = lv.flay[q];
    const FT* Fj = lv.F[q] + (long long)j * nb * r + o;
    const C* Xg = X + (long long)src * nb + o;
    const int mtr = rs / 4, mtk = ks / 4, nmt = mtr * mtk;
    const int G = max(1, 256 / nmt);
    const int mt = threadIdx.x % nmt, rg = threadIdx.x / nmt;
    const bool active = rg < G;
    const int t0 = (mt % mtr) * 4, c0 = (mt / mtr) * 4;
    C acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = czero<C>();
    // the next tile's loads are issued into registers before the current
    // tile's products (rs, ks <= 64: at most 8 entries of each per thread)
    C fpre[8], xpre[8];
    auto fetch = [&](int r0) {
        const int nr = min(TR, CH - r0);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = threadIdx.x + u * 256;
            const int cc = e / TR, rr = e - cc * TR;
            const FT* fp = flay == FAC_PLAIN ? Fj + (long long)cc * nb + r0 + rr
                                             : lv.F[q] + fac_index(flay, nb, r, lv.rp, j, o + r0 + rr, cc);
            fpre[u] = (e < TR * rs && rr < nr && cc < r) ? ldfac(fp) : czero<C>();
            xpre[u] = (e < TR * ks && rr < nr && cc < k) ? Xg[(long long)cc * m + r0 + rr] : czero<C>();
        }
    };
    fetch(0);
    for (int r0 = 0; r0 < CH; r0 += TR) {
        const int nr = min(TR, CH - r0);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = threadIdx.x + u * 256;
            const int cc = e / TR, rr = e - cc * TR;
            if (e < TR * rs) Fs[rr * fsd + cc] = fpre[u];
            if (e < TR * ks) Xs[rr * xsd + cc] = xpre[u];
        }
        __syncthreads();
        if (r0 + TR < CH) fetch(r0 + TR);
        if (active) {
            for (int rr = rg; rr < nr; rr += G) {
                C f[4], x[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) f[a] = Fs[rr * fsd + t0 + a];
#pragma unroll
                for (int b = 0; b < 4; ++b) x[b] = Xs[rr * xsd + c0 + b];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) cfmac(acc[a][b], f[a], x[b]);
            }
        }
        __syncthreads();
    }
    const int nout = r * k;
    if (active) {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b)
                if (t0 + a < r && c0 + b < k) Red[(long long)rg * nout + (c0 + b) * r + t0 + a] = acc[a][b];
    }
    __syncthreads();
    C* out = P + (long long)blockIdx.x * nout;
    for (int e = threadIdx.x; e < nout; e += 256) {
        C sacc = czero<C>();
        for (int g = 0; g < G; ++g) sacc = cadd(sacc, Red[(long long)g * nout + e]);
        out[e] = sacc;
    }
}

// T[level q][block j] = sum over the block's chunks of the partials, in order.
template <typename C, typename FT>
__global__ void k_lr_reduce(LrLevels<C, FT> lv, int r, int k, const C* __restrict__ P, C* __restrict__ T) {
    const long long nout = (long long)r * k;
    const long long tot = lv.t0[lv.nlev] * nout;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const long long tb = e / nout;
        const int oi = (int)(e - tb * nout);
        int q = 0;
        while (q + 1 < lv.nlev && tb >= lv.t0[q + 1]) ++q;
        const int j = (int)(tb - lv.t0[q]);
        const int per = lv.nb[q] / lv.ch[q];
        const C* p = P + ((long long)lv.chunk0[q] + (long long)j * per) * nout + oi;
        C s = czero<C>();
        for (int u = 0; u < per; ++u) s = cadd(s, p[(long long)u * nout]);
        T[e] = s;
    }
}

// Y[i][c] += sum over levels of G_b'(row) T_b': thread (4 consecutive rows,
// group of 8 columns); the 4 rows share their block at every level (block
// sizes are multiples of 4), so each T entry loaded serves 4 rows.
template <typename C, typename FT>
__global__ void __launch_bounds__(128)
k_lr_apply(LrLevels<C, FT> lv, int m, int r, int k, const C* __restrict__ T, int swapC, C* __restrict__ Y) {
    const int ngrp = (k + 7) / 8;
    const int slots = 128 / ngrp;
    const int slot = threadIdx.x % slots, g = threadIdx.x / slots;
    if (g >= ngrp) return;
    const int i0 = (blockIdx.x * slots + slot) * 4;
    if (i0 >= m) return;
    const int c0 = g * 8;
    const long long nout = (long long)r * k;
    // four factor columns' loads in flight (one for FP64, where registers run out)
    constexpr int UNR = sizeof(C) == 16 ? 1 : 4;
    C acc[4][8];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[a][u] = czero<C>();
    for (int q = 0; q < lv.nlev; ++q) {
        const int nb = lv.nb[q];
        const int b = i0 / nb, o = i0 - b * nb;
        const int bb = swapC ? (b ^ 1) : b;
        const int glay = lv.glay[q];
        const FT* Gb = lv.G[q] + (long long)bb * nb * r + o;
        const C* Tb = T + (lv.t0[q] + bb) * nout;
#pragma unroll UNR
        for (int t = 0; t < r; ++t) {
            C gv[4], tv[8];
#pragma unroll
            for (int a = 0; a < 4; ++a)
                gv[a] = ldfac(glay == FAC_PLAIN ? Gb + (long long)t * nb + a
                                                : lv.G[q] + fac_index(glay, nb, r, lv.rp, bb, o + a, t));
#pragma unroll
            for (int u = 0; u < 8; ++u) tv[u] = c0 + u < k ? Tb[(long long)(c0 + u) * r + t] : czero<C>();
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int u = 0; u < 8; ++u) cfma(acc[a][u], gv[a], tv[u]);
        }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
        if (c0 + u < k) {
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                C* y = Y + (long long)(c0 + u) * m + i0 + a;
                *y = cadd(*y, acc[a][u]);
            }
        }
}

// The three launches of the fused level products for a prepared level list.
template <typename C, typename FT>
lsw_status lr_launch(const LrLevels<C, FT>& lv, int m, int r, int k, const C* X, C* Y, int swapA, int swapC,
                     cudaStream_t st) {
    const long long nout = (long long)r * k;
    DevBuf P, T;
    LSW_TRY(P.alloc(sizeof(C) * (size_t)lv.chunk0[lv.nlev] * nout, st));
    LSW_TRY(T.alloc(sizeof(C) * (size_t)lv.t0[lv.nlev] * nout, st));
    static std::atomic<bool> attr{false};
    if (!attr.load()) {
        LSW_CUDA(cudaFuncSetAttribute(k_lr_partial<C, FT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        attr.store(true);
    }
    const int rs = (r + 3) & ~3, ks = (k + 3) & ~3;
    const int Gr = std::max(1, 256 / ((rs / 4) * (ks / 4)));
    const size_t smem = sizeof(C) * (32 * (size_t)(rs + ks + 2) + (size_t)Gr * r * k);
    // both factors of every level once, X once per level, Y read and written
    KTimer kt("lr_levels", st, (double)lv.nlev * m * (2.0 * r * sizeof(FT) + (double)k * sizeof(C)) + 2.0 * m * k * sizeof(C),
              8.0 * 2.0 * lv.nlev * (double)m * r * k);
    // BF16 factors and complex64 vectors: on the tensor cores when the shapes allow
    bool tc = false;
    if constexpr (std::is_same<C, float2>::value && std::is_same<FT, uint32_t>::value) tc = lr_tc_fits(lv, m, r, k);
    {
        // every level's first factor once and X once per level
        KTimer ktp("lr_partial", st, (double)lv.nlev * m * ((double)r * sizeof(FT) + (double)k * sizeof(C)),
                   8.0 * lv.nlev * (double)m * r * k);
        if (tc) {
            if constexpr (std::is_same<C, float2>::value && std::is_same<FT, uint32_t>::value)
                LSW_TRY(lr_partial_tc(lv, m, r, k, X, swapA, P.as<C>(), st));
        } else {
            k_lr_partial<C, FT><<<lv.chunk0[lv.nlev], 256, smem, st>>>(lv, m, r, k, X, swapA, P.as<C>());
            LSW_LAUNCH_CHECK();
        }
    }
    {
        KTimer ktr("lr_reduce", st, sizeof(C) * (double)(lv.chunk0[lv.nlev] + lv.t0[lv.nlev]) * nout, 0.0);
        k_lr_reduce<C, FT><<<gridn(lv.t0[lv.nlev] * nout), 256, 0, st>>>(lv, r, k, P.as<C>(), T.as<C>());
        LSW_LAUNCH_CHECK();
    }
    // every level's second factor once, Y read and written
    KTimer kta("lr_apply", st, (double)lv.nlev * m * r * sizeof(FT) + 2.0 * m * k * sizeof(C),
               8.0 * lv.nlev * (double)m * r * k);
    if (tc) {
        if constexpr (std::is_same<C, float2>::value && std::is_same<FT, uint32_t>::value)
            return lr_apply_tc(lv, m, r, k, T.as<C>(), swapC, Y, st);
    }
    const int rows_cta = 4 * (128 / ((k + 7) / 8));
    k_lr_apply<C, FT><<<(m + rows_cta - 1) / rows_cta, 128, 0, st>>>(lv, m, r, k, T.as<C>(), swapC, Y);
    LSW_LAUNCH_CHECK();
    return LSW_OK;
}

// Shapes the fused kernels take: k <= 64 columns, rank <= 64, r k <= 4096,
// block sizes (hence node sizes) multiples of 4.
template <typename R>
bool lr_fused_ok(const HStore<R>& H, int l, int k) {
    return k >= 1 && k <= 64 && H.r <= 64 && H.r * k <= 4096 && (H.nl(H.L) & 3) == 0 && H.L - l <= kMaxLev;
}

// Levels l+1..L of node (l, c): F and G are U or W (see the callers).
template <typename R>
lsw_status lr_levels(const HStore<R>& H, int l, int c, bool F_is_W, const typename Cx<R>::T* X, int k,
                     typename Cx<R>::T* Y, int swapA, int swapC, cudaStream_t st) {
    typedef typename Cx<R>::T C;
    const int L = H.L, r = H.r, m = H.nl(l);
    if (L - l > kMaxLev) return LSW_ERR_UNSUPPORTED_SIZE;
    if (L <= l) return LSW_OK;
    if (r * k > 4096 || k > 64 || r > 64 || (m & 3)) return LSW_ERR_INVALID_ARG;
    LrLevels<C, C> lv;
    lv.nlev = L - l;
    lv.chunk0[0] = 0;
    lv.t0[0] = 0;
    for (int q = 0; q < lv.nlev; ++q) {
        const int lp = l + 1 + q, cnt = 1 << (lp - l), nb = H.nl(lp);
        const size_t first = (size_t)c * cnt;
        const C* U0 = H.U[lp] + first * nb * r;
        const C* W0 = H.W[lp] + first * nb * r;
        lv.F[q] = F_is_W ? W0 : U0;
        lv.G[q] = F_is_W ? U0 : W0;
        lv.nb[q] = nb;
        lv.ch[q] = std::min(nb, 1024);
        lv.chunk0[q + 1] = lv.chunk0[q] + m / lv.ch[q];
        lv.t0[q + 1] = lv.t0[q] + cnt;
    }
    for (int q = lv.nlev; q < kMaxLev; ++q) {
        lv.F[q] = lv.G[q] = nullptr;
        lv.nb[q] = lv.ch[q] = 1;
        lv.chunk0[q + 1] = lv.chunk0[q];
        lv.t0[q + 1] = lv.t0[q];
    }
    return lr_launch<C, C>(lv, m, r, k, X, Y, swapA, swapC, st);
}

// Y_b = D_b X_b for nleaf consecutive dense leaves (nL x nL each) and k
// columns (X, Y: ld m): on the tensor cores in FP32 when the shape allows.
template <typename R>
lsw_status leaf_product(const typename Cx<R>::T* D0, int nL, const typename Cx<R>::T* X, int m, int k,
                        typename Cx<R>::T* Y, int nleaf, cudaStream_t st) {
    typedef typename Cx<R>::T C;
    return gemm<R>('N', 'N', nL, k, nL, one<C>(), D0, nL, (long long)nL * nL, X, m, nL, zero<C>(), Y, m, nL, nleaf, st);
}

template <>
lsw_status leaf_product<float>(const float2* D0, int nL, const float2* X, int m, int k, float2* Y, int nleaf,
                               cudaStream_t st) {
    if (tc_gemm_enabled() && tc_gemm_fits(nL, k, nL))
        return cgemm_tc(D0, nL, (long long)nL * nL, X, m, nL, Y, m, nL, nL, k, nL, make_float2(1.f, 0.f), nleaf, st);
    return gemm<float>('N', 'N', nL, k, nL, one<float2>(), D0, nL, (long long)nL * nL, X, m, nL, zero<float2>(), Y, m,
                       nL, nleaf, st);
}

// Y = X_sub * Xin for node (l, c) (k columns, ld = n_l); T: workspace of
// 2^(L-l) * r * k complex (used by the per-level path for k > 64).
template <typename R>
lsw_status hmv(const HStore<R>& H, int l, int c, const typename Cx<R>::T* X, int k, typename Cx<R>::T* Y,
               typename Cx<R>::T* T, cudaStream_t st) {
    typedef typename Cx<R>::T C;
    const int m = H.nl(l), L = H.L, r = H.r, nL = H.nl(L);
    const int nleaf = 1 << (L - l);
    const C* D0 = H.D + (size_t)c * nleaf * nL * nL;
    LSW_TRY(leaf_product<R>(D0, nL, X, m, k, Y, nleaf, st));
    // T_j = W_j^H X[sibling rows];  Y[rows j] += U_j T_j
    if (lr_fused_ok(H, l, k)) return lr_levels<R>(H, l, c, true, X, k, Y, 1, 0, st);
    for (int lp = l + 1; lp <= L; ++lp) {
        const int cnt = 1 << (lp - l), nb = H.nl(lp);
        const size_t first = (size_t)c * cnt;
        const C* U0 = H.U[lp] + first * nb * r;
        const C* W0 = H.W[lp] + first * nb * r;
        LSW_TRY(gemm<R>('C', 'N', r, k, nb, one<C>(), W0, nb, 2LL * nb * r, X + nb, m, 2LL * nb, zero<C>(), T, r,
                        2LL * r * k, cnt / 2, st));
        LSW_TRY(gemm<R>('C', 'N', r, k, nb, one<C>(), W0 + (size_t)nb * r, nb, 2LL * nb * r, X, m, 2LL * nb, zero<C>(),
                        T + (size_t)r * k, r, 2LL * r * k, cnt / 2, st));
        LSW_TRY(gemm<R>('N', 'N', nb, k, r, one<C>(), U0, nb, (long long)nb * r, T, r, (long long)r * k, one<C>(), Y, m,
                        nb, cnt, st));
    }
    return LSW_OK;
}

// Y = X_sub^H * Xin for node (l, c).
template <typename R>
lsw_status hmv_adj(const HStore<R>& H, int l, int c, const typename Cx<R>::T* X, int k, typename Cx<R>::T* Y,
                   typename Cx<R>::T* T, cudaStream_t st) {
    typedef typename Cx<R>::T C;
    const int m = H.nl(l), L = H.L, r = H.r, nL = H.nl(L);
    const int nleaf = 1 << (L - l);
    const C* D0 = H.D + (size_t)c * nleaf * nL * nL;
    LSW_TRY(gemm<R>('C', 'N', nL, k, nL, one<C>(), D0, nL, (long long)nL * nL, X, m, nL, zero<C>(), Y, m, nL, nleaf, st));
    // T_j = U_j^H X[rows j];  Y[rows j ^ 1] += W_j T_j
    if (lr_fused_ok(H, l, k)) return lr_levels<R>(H, l, c, false, X, k, Y, 0, 1, st);
    for (int lp = l + 1; lp <= L; ++lp) {
        const int cnt = 1 << (lp - l), nb = H.nl(lp);
        const size_t first = (size_t)c * cnt;
        const C* U0 = H.U[lp] + first * nb * r;
        const C* W0 = H.W[lp] + first * nb * r;
        LSW_TRY(gemm<R>('C', 'N', r, k, nb, one<C>(), U0, nb, (long long)nb * r, X, m, nb, zero<C>(), T, r,
                        (long long)r * k, cnt, st));
        LSW_TRY(gemm<R>('N', 'N', nb, k, r, one<C>(), W0, nb, 2LL * nb * r, T, r, 2LL * r * k, one<C>(), Y + nb, m,
                        2LL * nb, cnt / 2, st));
        LSW_TRY(gemm<R>('N', 'N', nb, k, r, one<C>(), W0 + (size_t)nb * r, nb, 2LL * nb * r, T + (size_t)r * k, r,
                        2LL * r * k, one<C>(), Y, m, 2LL * nb, cnt / 2, st));
    }
    return LSW_OK;
}

// Node (l, c) of M += X Y^H (X, Y: n_l x r), every off-diagonal block cut
// back to rank r by Algorithm 1 (q = 0) through its factors.
template <typename R>
lsw_status add_lowrank(HStore<R>& M, int l, int c, const typename Cx<R>::T* X, const typename Cx<R>::T* Y, int op,
                       int call_l, int call_c, int oversample, uint64_t seed, cudaStream_t st0,
                       LeafUpd<R>* lu = nullptr) {
    KTimer kt_all("hodlr_add_lowrank", st0, 0, 0);
    cudaStream_t st = st0;
    typedef typename Cx<R>::T C;
    const int m = M.nl(l), L = M.L, r = M.r, nL = M.nl(L);
    const int rp = r + oversample;
    const int nleaf = 1 << (L - l);
    if (lu) {
        // the leaves hold inverses: each leaf j of the node gets
        // D_j^-1 <- (D_j + U_j V_j^H)^-1 with U_j, V_j its rows of X, Y, by
        // Woodbury, batched over the node's leaves:
        //   D^-1 - (D^-1 U) (I + V^H D^-1 U)^-1 (V^H D^-1)
        KTimer kt_leaf("hodlr_leaf_woodbury", st, 0, 0);
        LSW_TRY(lu->wait(c * nleaf + nleaf - 1, st));
        C* D0 = M.D + (size_t)c * nleaf * nL * nL;
        const long long nn = (long long)nL * nL, nr = (long long)nL * r;
        DevBuf T1, T2, T3, Mc;
        LSW_TRY(T1.alloc(sizeof(C) * (size_t)nleaf * nr, st));
        LSW_TRY(T2.alloc(sizeof(C) * (size_t)nleaf * nr, st));
        LSW_TRY(T3.alloc(sizeof(C) * (size_t)nleaf * nr, st));
        LSW_TRY(Mc.alloc(sizeof(C) * (size_t)nleaf * r * r, st));
        // T1 = D^-1 U, T2 = V^H D^-1, Mc = I + V^H T1
        LSW_TRY(gemm<R>('N', 'N', nL, r, nL, one<C>(), D0, nL, nn, X, m, nL, zero<C>(), T1.as<C>(), nL, nr, nleaf, st));
        LSW_TRY(gemm<R>('C', 'N', r, nL, nL, one<C>(), Y, m, nL, D0, nL, nn, zero<C>(), T2.as<C>(), r, nr, nleaf, st));
        LSW_TRY(gemm<R>('C', 'N', r, r, nL, one<C>(), Y, m, nL, T1.as<C>(), nL, nr, zero<C>(), Mc.as<C>(), r,
                        (long long)r * r, nleaf, st));
        k_eye_plus<C><<<gridn((long long)r * nleaf), 256, 0, st>>>(Mc.as<C>(), r, nleaf);
        LSW_LAUNCH_CHECK();
        LSW_TRY(inverse_gj<R>(Mc.as<C>(), r, (long long)r * r, nleaf, st));
        // T3 = Mc^-1 T2, D^-1 -= T1 T3
        LSW_TRY(gemm<R>('N', 'N', r, nL, r, one<C>(), Mc.as<C>(), r, (long long)r * r, T2.as<C>(), r, nr, zero<C>(),
                        T3.as<C>(), r, nr, nleaf, st));
        LSW_TRY(gemm<R>('N', 'N', nL, nL, r, minus_one<C>(), T1.as<C>(), nL, nr, T3.as<C>(), r, nr, one<C>(), D0, nL, nn,
                        nleaf, st));
    } else {
        C* D0 = M.D + (size_t)c * nleaf * nL * nL;
        LSW_TRY(gemm<R>('N', 'C', nL, nL, r, one<C>(), X, m, nL, Y, m, nL, one<C>(), D0, nL, (long long)nL * nL, nleaf,
                        st));
    }
    Fork fk(st0);
    for (int lp = l + 1; lp <= L; ++lp) {
        // the levels' recompressions are independent of each other
        cudaStream_t st = fk.child(lp);
        const int cnt = 1 << (lp - l), nb = M.nl(lp);
        const size_t first = (size_t)c * cnt;
        C* U0 = M.U[lp] + first * nb * r;
        C* W0 = M.W[lp] + first * nb * r;
        DevBuf uc, wc, om, tt, ys, yt, dw2, dw3;
        const size_t cat = (size_t)cnt * nb * 2 * r, pro = (size_t)cnt * nb * rp;
        LSW_TRY(uc.alloc(sizeof(C) * cat, st));
        LSW_TRY(wc.alloc(sizeof(C) * cat, st));
        LSW_TRY(om.alloc(sizeof(C) * pro, st));
        LSW_TRY(ys.alloc(sizeof(C) * pro, st));
        LSW_TRY(yt.alloc(sizeof(C) * pro, st));
        LSW_TRY(tt.alloc(sizeof(C) * (size_t)cnt * 2 * r * rp, st));
        k_concat<C><<<gridn((long long)cat), 256, 0, st>>>(U0, W0, X, Y, nb, r, m, cnt, uc.as<C>(), wc.as<C>());
        LSW_LAUNCH_CHECK();
        std::vector<uint32_t> w2(cnt, stream_w2(TAG_RECOMPRESS, op, call_l, call_c)), w3(cnt);
        for (int j = 0; j < cnt; ++j) w3[j] = ((uint32_t)lp << 16) | (uint32_t)(first + j);
        LSW_TRY(upload(dw2, w2, st));
        LSW_TRY(upload(dw3, w3, st));
        LSW_TRY(gaussian_fill<R>(om.as<C>(), nb, rp, (long long)nb * rp, cnt, seed, dw2.as<uint32_t>(),
                                 dw3.as<uint32_t>(), st));
        const long long sc = (long long)nb * 2 * r, sp = (long long)nb * rp, stt = 2LL * r * rp;
        // Y = Uc (Wc^H Omega)
        LSW_TRY(gemm<R>('C', 'N', 2 * r, rp, nb, one<C>(), wc.as<C>(), nb, sc, om.as<C>(), nb, sp, zero<C>(), tt.as<C>(),
                        2 * r, stt, cnt, st));
        LSW_TRY(gemm<R>('N', 'N', nb, rp, 2 * r, one<C>(), uc.as<C>(), nb, sc, tt.as<C>(), 2 * r, stt, zero<C>(),
                        ys.as<C>(), nb, sp, cnt, st));
        LSW_TRY(qr_sketch<R>(ys.as<C>(), nb, rp, sp, cnt, st));
        // Yt = Wc (Uc^H Q)
        LSW_TRY(gemm<R>('C', 'N', 2 * r, rp, nb, one<C>(), uc.as<C>(), nb, sc, ys.as<C>(), nb, sp, zero<C>(), tt.as<C>(),
                        2 * r, stt, cnt, st));
        LSW_TRY(gemm<R>('N', 'N', nb, rp, 2 * r, one<C>(), wc.as<C>(), nb, sc, tt.as<C>(), 2 * r, stt, zero<C>(),
                        yt.as<C>(), nb, sp, cnt, st));
        LSW_TRY(truncate<R>(ys.as<C>(), nb, yt.as<C>(), nb, rp, r, cnt, one<C>(), U0, (long long)nb * r, W0,
                            (long long)nb * r, st));
    }
    return fk.join();
}

// Inverse of node (l, c) of X written into the same node of Hi (recursive
// block inversion).  X's node c+1 subtree is overwritten by the Schur
// complement S = D - C A^-1 B.
template <typename R>
lsw_status invert_node(HStore<R>& X, int l, int c, HStore<R>& Hi, int oversample, uint64_t seed, cudaStream_t st,
                       LeafUpd<R>& lu) {
    typedef typename Cx<R>::T C;
    const int L = X.L, r = X.r;
    if (l == L) {
        // X's leaf already holds the inverse of the leaf to invert (the
        // original leaf's inverse with every update of its ancestors' Schur
        // complements folded in)
        const int nL = X.nl(L);
        const long long nn = (long long)nL * nL;
        LSW_TRY(lu.wait(c, st));
        LSW_CUDA(cudaMemcpyAsync(Hi.D + (size_t)c * nn, X.D + (size_t)c * nn, sizeof(C) * nn, cudaMemcpyDeviceToDevice,
                                 st));
        return LSW_OK;
    }
    const int a = 2 * c, b = 2 * c + 1, m1 = X.nl(l + 1);
    const int nb1 = m1 * r;
    C* UB = X.U[l + 1] + (size_t)a * nb1;   // B = UB WB^H
    C* WB = X.W[l + 1] + (size_t)a * nb1;
    C* UC = X.U[l + 1] + (size_t)b * nb1;   // C = UC WC^H
    C* WC = X.W[l + 1] + (size_t)b * nb1;
    LSW_TRY(invert_node<R>(X, l + 1, a, Hi, oversample, seed, st, lu));
    // the first use of level l + 1's blocks (deeper levels were waited for
    // inside the subtree just inverted, which holds a node of every level)
    LSW_TRY(lu.wait_level(l + 1, st));
    DevBuf P, Rm, T1, T2, K, XK, T;
    const size_t vb = sizeof(C) * (size_t)m1 * r;
    LSW_TRY(P.alloc(vb, st));
    LSW_TRY(Rm.alloc(vb, st));
    LSW_TRY(T1.alloc(vb, st));
    LSW_TRY(T2.alloc(vb, st));
    LSW_TRY(XK.alloc(vb, st));
    LSW_TRY(K.alloc(sizeof(C) * r * r, st));
    LSW_TRY(T.alloc(sizeof(C) * ((size_t)1 << (L - l)) * r * r, st));
    {
        KTimer kt_sub("hodlr_subtree_products", st, 0, 0);
        LSW_TRY(hmv<R>(Hi, l + 1, a, UB, r, P.as<C>(), T.as<C>(), st));        // P = A^-1 UB
        LSW_TRY(hmv_adj<R>(Hi, l + 1, a, WC, r, Rm.as<C>(), T.as<C>(), st));   // R = A^-H WC
    }
    LSW_TRY(gemm<R>('C', 'N', r, r, m1, one<C>(), WC, m1, 0, P.as<C>(), m1, 0, zero<C>(), K.as<C>(), r, 0, 1, st));
    // S = D - UC K WB^H  (in place on X's node b)
    LSW_TRY(gemm<R>('N', 'N', m1, r, r, minus_one<C>(), UC, m1, 0, K.as<C>(), r, 0, zero<C>(), XK.as<C>(), m1, 0, 1, st));
    LSW_TRY(add_lowrank<R>(X, l + 1, b, XK.as<C>(), WB, 0, l, c, oversample, seed, st, &lu));
    LSW_TRY(invert_node<R>(X, l + 1, b, Hi, oversample, seed, st, lu));     // S^-1 into Hi
    {
        KTimer kt_sub("hodlr_subtree_products", st, 0, 0);
        LSW_TRY(hmv<R>(Hi, l + 1, b, UC, r, T1.as<C>(), T.as<C>(), st));       // T1 = S^-1 UC
        LSW_TRY(hmv_adj<R>(Hi, l + 1, b, WB, r, T2.as<C>(), T.as<C>(), st));   // T2 = S^-H WB
    }
    LSW_TRY(gemm<R>('C', 'N', r, r, m1, one<C>(), WB, m1, 0, T1.as<C>(), m1, 0, zero<C>(), K.as<C>(), r, 0, 1, st));
    // top-left: A^-1 + P K2 R^H
    LSW_TRY(gemm<R>('N', 'N', m1, r, r, one<C>(), P.as<C>(), m1, 0, K.as<C>(), r, 0, zero<C>(), XK.as<C>(), m1, 0, 1, st));
    LSW_TRY(add_lowrank<R>(Hi, l + 1, a, XK.as<C>(), Rm.as<C>(), 1, l, c, oversample, seed, st));
    // off-diagonal blocks of the inverse: -P T2^H and -T1 R^H
    const long long nn = (long long)m1 * r;
    k_scale_copy<C><<<gridn(nn), 256, 0, st>>>(P.as<C>(), Hi.U[l + 1] + (size_t)a * nb1, nn, (R)-1);
    LSW_LAUNCH_CHECK();
    k_scale_copy<C><<<gridn(nn), 256, 0, st>>>(T2.as<C>(), Hi.W[l + 1] + (size_t)a * nb1, nn, (R)1);
    LSW_LAUNCH_CHECK();
    k_scale_copy<C><<<gridn(nn), 256, 0, st>>>(T1.as<C>(), Hi.U[l + 1] + (size_t)b * nb1, nn, (R)-1);
    LSW_LAUNCH_CHECK();
    k_scale_copy<C><<<gridn(nn), 256, 0, st>>>(Rm.as<C>(), Hi.W[l + 1] + (size_t)b * nb1, nn, (R)1);
    LSW_LAUNCH_CHECK();
    return LSW_OK;
}

// ------------------------------------------------------------ full builds
template <typename R>
lsw_status build_hodlr(const lsw_green* g, const double* chi, const lsw_hparams* hp, lsw_hmatrix* h, cudaStream_t st,
                       HStore<R>& Hi) {
    typedef typename Cx<R>::T C;
    const Tree& tr = h->tree;
    const int L = hp->levels, r = hp->rank, rp = hp->rank + hp->oversample;
    HStore<R> X;
    struct Rel { HStore<R>* s; ~Rel() { s->release(); } } rel{&X};
    LSW_TRY(X.alloc(L, r, tr.n));
    // one spectrum per level (the parent boxes of a level share one shape)
    std::vector<Spectrum> spec(L + 1);
    struct SpecGuard {
        std::vector<Spectrum>* v;
        ~SpecGuard() { for (auto& s : *v) free_spectrum(&s); }
    } specguard{&spec};
    for (int l = 1; l <= L; ++l) {
        const int4 P0 = tr.node(l - 1, 0);
        LSW_TRY(build_spectrum(g, P0.y - P0.x, P0.w - P0.z, &spec[l], st));
    }
    const int nL = tr.nl(L);
    const int nleaf = 1 << L;
    LeafUpd<R> lu;
    struct EvGuard {
        std::vector<cudaEvent_t>* v;
        ~EvGuard() { for (auto e : *v) cudaEventDestroy(e); }
    } evguard{&lu.ready};
    // The original leaves are inverted on their own stream, in batches in
    // the order the recursive inversion first needs them (leaf 0 first): the
    // first eighth, the next eighth, the next quarter, the last half.  Each
    // batch fires an event that the inversion waits on before its first use
    // of a leaf of that batch, so later batches overlap the inversion.
    {
        const int b0 = std::max(1, nleaf / 8);
        for (int e = b0; e < nleaf; e *= 2) lu.end.push_back(e);
        lu.end.push_back(nleaf);
        for (size_t b = 0; b < lu.end.size(); ++b) {
            cudaEvent_t ev;
            LSW_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            lu.ready.push_back(ev);
        }
    }
    Fork fkd(st);
    {
        cudaStream_t sd = fkd.child(0);
        KTimer kt("hodlr_leaf_inverse", sd, 0, 0);
        k_leaf_assemble<C><<<gridn((long long)tr.n * nL), 256, 0, sd>>>(g->table, g->nz, chi, h->perm_d, nL, nleaf, X.D);
        LSW_LAUNCH_CHECK();
        int first = 0;
        for (size_t b = 0; b < lu.end.size(); ++b) {
            const long long nn = (long long)nL * nL;
            LSW_TRY(inverse_gj<R>(X.D + (size_t)first * nn, nL, nn, lu.end[b] - first, sd));
            LSW_CUDA(cudaEventRecord(lu.ready[b], sd));
            first = lu.end[b];
        }
    }
    // The levels are independent of each other and of the dense leaves:
    // sketch them concurrently, each on a stream of its own, deepest first;
    // the inversion starts at once and waits for a level only where it
    // first reads it (the recursion reaches the deep levels first).
    std::vector<cudaStream_t> lstream(L + 1, nullptr);
    struct LevelGuard {
        std::vector<cudaStream_t>* s;
        std::vector<cudaEvent_t>* e;
        ~LevelGuard() {
            for (auto v : *e) if (v) cudaEventDestroy(v);
            for (auto v : *s) if (v) cudaStreamDestroy(v);
        }
    } levelguard{&lstream, &lu.level_done};
    lu.level_done.assign(L + 1, nullptr);
    {
        cudaEvent_t begin;
        LSW_CUDA(cudaEventCreateWithFlags(&begin, cudaEventDisableTiming));
        LSW_CUDA(cudaEventRecord(begin, st));
        for (int l = L; l >= 1; --l) {
            LSW_CUDA(cudaStreamCreateWithFlags(&lstream[l], cudaStreamNonBlocking));
            LSW_CUDA(cudaStreamWaitEvent(lstream[l], begin, 0));
            {
                KTimer kt("hodlr_level_sketch", lstream[l], 0, 0);
                LSW_TRY(build_level<R>(g, chi, tr, l, r, rp, hp->q, hp->seed, X, spec[l], lstream[l]));
            }
            LSW_CUDA(cudaEventCreateWithFlags(&lu.level_done[l], cudaEventDisableTiming));
            LSW_CUDA(cudaEventRecord(lu.level_done[l], lstream[l]));
        }
        cudaEventDestroy(begin);
    }
    KTimer kti("hodlr_invert", st, 0, 0);
    LSW_TRY(Hi.alloc(L, r, tr.n));
    LSW_TRY(invert_node<R>(X, 0, 0, Hi, hp->oversample, hp->seed, st, lu));
    for (int l = 1; l <= L; ++l) LSW_TRY(lu.wait_level(l, st));
    LSW_TRY(fkd.join());
    LSW_CUDA(cudaStreamSynchronize(st));
    return LSW_OK;
}

// Sketch (G0 V)[s, t] ~ U W^H for boxes s, t inside the grid (strip order
// inside each box).  alphaU scales U.
template <typename R>
lsw_status sketch_boxes(const lsw_green* g, const double* chi, lsw_box s, lsw_box t, int r, int oversample, int q,
                        uint64_t seed, uint32_t w2v, uint32_t w3v, typename Cx<R>::T alphaU, typename Cx<R>::T* U,
                        typename Cx<R>::T* W, cudaStream_t st) {
    typedef typename Cx<R>::T C;
    const int rp = r + oversample;
    lsw_box B{std::min(s.z0, t.z0), std::max(s.z1, t.z1), std::min(s.x0, t.x0), std::max(s.x1, t.x1)};
    if (!is_pow2(B.z1 - B.z0) || !is_pow2(B.x1 - B.x0)) B = lsw_box{0, g->nz, 0, g->nx};
    const int bz = B.z1 - B.z0, bx = B.x1 - B.x0;
    const long long boxn = (long long)bz * bx;
    const int ns = (s.z1 - s.z0) * (s.x1 - s.x0), nt = (t.z1 - t.z0) * (t.x1 - t.x0);
    auto mapof = [&](lsw_box q_) {
        std::vector<int> m;
        for (int ix = q_.x0; ix < q_.x1; ++ix)
            for (int iz = q_.z0; iz < q_.z1; ++iz) m.push_back((ix - B.x0) * bz + (iz - B.z0));
        return m;
    };
    Spectrum sp;
    const bool full = (bz == g->nz && bx == g->nx);
    if (!full) LSW_TRY(build_spectrum(g, bz, bx, &sp, st));
    struct SpGuard { Spectrum* s; bool own; ~SpGuard() { if (own) free_spectrum(s); } } guard{&sp, !full};
    const Spectrum& spec = full ? g->full : sp;
    DevBuf ms, mt, dorg, dw2, dw3, om, qb, yt, vin, vout, work;
    LSW_TRY(upload(ms, mapof(s), st));
    LSW_TRY(upload(mt, mapof(t), st));
    LSW_TRY(upload(dorg, std::vector<int2>{make_int2(B.z0, B.x0)}, st));
    LSW_TRY(upload(dw2, std::vector<uint32_t>{w2v}, st));
    LSW_TRY(upload(dw3, std::vector<uint32_t>{w3v}, st));
    LSW_TRY(om.alloc(sizeof(C) * (size_t)nt * rp, st));
    LSW_TRY(qb.alloc(sizeof(C) * (size_t)ns * rp, st));
    LSW_TRY(yt.alloc(sizeof(C) * (size_t)nt * rp, st));
    LSW_TRY(vin.alloc(sizeof(C) * rp * boxn, st));
    LSW_TRY(vout.alloc(sizeof(C) * rp * boxn, st));
    LSW_TRY(work.alloc(sizeof(C) * rp * boxn * 2, st));
    LSW_TRY(gaussian_fill<R>(om.as<C>(), nt, rp, (long long)nt * rp, 1, seed, dw2.as<uint32_t>(), dw3.as<uint32_t>(), st));
    OpGeom geo{bz, bx, chi, g->nz, dorg.as<int2>(), rp};
    auto fwd = [&](const C* X, C* Y) -> lsw_status {
        LSW_CUDA(cudaMemsetAsync(vin.p, 0, sizeof(C) * rp * boxn, st));
        k_scatter_map<C><<<gridn((long long)nt * rp), 256, 0, st>>>(X, nt, rp, mt.as<int>(), boxn, vin.as<C>());
        LSW_LAUNCH_CHECK();
        LSW_TRY(op_apply<R>(g, spec, geo, LSW_OP_PLAIN, vin.as<C>(), nullptr, vout.as<C>(), rp, work.as<C>(), st));
        k_gather_map<C><<<gridn((long long)ns * rp), 256, 0, st>>>(vout.as<C>(), ns, rp, ms.as<int>(), boxn, Y);
        LSW_LAUNCH_CHECK();
        return LSW_OK;
    };
    auto adj = [&](const C* X, C* Y) -> lsw_status {
        LSW_CUDA(cudaMemsetAsync(vin.p, 0, sizeof(C) * rp * boxn, st));
        k_scatter_map<C><<<gridn((long long)ns * rp), 256, 0, st>>>(X, ns, rp, ms.as<int>(), boxn, vin.as<C>());
        LSW_LAUNCH_CHECK();
        LSW_TRY(op_apply<R>(g, spec, geo, LSW_OP_ADJOINT, vin.as<C>(), nullptr, vout.as<C>(), rp, work.as<C>(), st));
        k_gather_map<C><<<gridn((long long)nt * rp), 256, 0, st>>>(vout.as<C>(), nt, rp, mt.as<int>(), boxn, Y);
        LSW_LAUNCH_CHECK();
        return LSW_OK;
    };
    LSW_TRY((range_finder<R>(ns, nt, rp, q, 1, om.as<C>(), qb.as<C>(), yt.as<C>(), fwd, adj, st)));
    LSW_TRY(truncate<R>(qb.as<C>(), ns, yt.as<C>(), nt, rp, r, 1, alphaU, U, (long long)ns * r, W, (long long)nt * r, st));
    LSW_CUDA(cudaStreamSynchronize(st));
    return LSW_OK;
}

template <typename R>
lsw_status build_smw(const lsw_green* g, const double* chi, const lsw_hparams* hp, lsw_hmatrix* h, cudaStream_t st) {
    typedef typename Cx<R>::T C;
    const int n = h->n, r = hp->rank;
    LSW_CUDA(cudaMalloc(&h->smwU, sizeof(C) * (size_t)n * r));
    LSW_CUDA(cudaMalloc(&h->smwW, sizeof(C) * (size_t)n * r));
    LSW_CUDA(cudaMalloc(&h->smwZ, sizeof(C) * (size_t)r * r));
    h->bytes = sizeof(C) * ((size_t)2 * n * r + (size_t)r * r);
    C* U = (C*)h->smwU;
    C* W = (C*)h->smwW;
    C* Z = (C*)h->smwZ;
    lsw_box all{0, g->nz, 0, g->nx};
    LSW_TRY(sketch_boxes<R>(g, chi, all, all, r, hp->oversample, hp->q, hp->seed, stream_w2(TAG_GLOBAL, 0, 0, 0), 0,
                            one<C>(), U, W, st));
    // Z = (I_r - W^H U)^-1   (Eq. 12)
    LSW_TRY(gemm<R>('C', 'N', r, r, n, one<C>(), W, n, 0, U, n, 0, zero<C>(), Z, r, 0, 1, st));
    k_eye_minus<C><<<1, 256, 0, st>>>(Z, r);
    LSW_LAUNCH_CHECK();
    LSW_TRY(inverse_gj<R>(Z, r, (long long)r * r, 1, st));
    LSW_CUDA(cudaStreamSynchronize(st));
    return LSW_OK;
}

// A level's factor (blocks of nb x r, column-major) into BF16 pairs in the
// storage lay (FAC_*), rp columns per block (the columns beyond r zero).
__global__ void k_to_bf16_fac(const float2* __restrict__ src, uint32_t* __restrict__ dst, int lay, int nb, int r,
                              int rp, long long nblk) {
    const long long tot = nblk * nb * rp;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const long long j = e / ((long long)nb * rp);
        const long long q = e - j * nb * rp;
        const int i = (int)(q / nb), o = (int)(q - (long long)i * nb);
        const float2 v = i < r ? src[(j * r + i) * nb + o] : make_float2(0.f, 0.f);
        const __nv_bfloat162 b = __floats2bfloat162_rn(v.x, v.y);
        dst[fac_index(lay, nb, r, rp, (int)j, o, i)] = *reinterpret_cast<const uint32_t*>(&b);
    }
}

__global__ void k_to_bf16(const float2* __restrict__ src, uint32_t* __restrict__ dst, long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const __nv_bfloat162 v = __floats2bfloat162_rn(src[e].x, src[e].y);
        dst[e] = *reinterpret_cast<const uint32_t*>(&v);
    }
}

// Y_b = D_b X_b with BF16 leaves on the CUDA cores (when the tensor-core
// kernel does not take the shape or is switched off): thread per output.
__global__ void k_leaf_bf16(const uint32_t* __restrict__ D, const float2* __restrict__ X, float2* __restrict__ Y,
                            int nL, int nleaf, int k, int ld) {
    const long long tot = (long long)nL * nleaf * k;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % nL);
        const long long rest = e / nL;
        const int b = (int)(rest % nleaf), j = (int)(rest / nleaf);
        const uint32_t* Db = D + (size_t)b * nL * nL;
        const float2* x = X + (size_t)j * ld + (size_t)b * nL;
        float2 acc = make_float2(0.f, 0.f);
        for (int t = 0; t < nL; ++t) cfma(acc, ldfac(Db + (size_t)t * nL + i), x[t]);
        Y[(size_t)j * ld + (size_t)b * nL + i] = acc;
    }
}

lsw_status to_bf16(const HStore<float>& H, HStoreB& B, cudaStream_t st) {
    // the product on this storage runs on the fused level kernels only
    if (H.L > kMaxLev || H.r > 64 || (H.L >= 1 && (H.nl(H.L) & 3))) return LSW_ERR_UNSUPPORTED_SIZE;
    B.L = H.L;
    B.r = H.r;
    B.n = H.n;
    const int nL = H.nl(H.L);
    const long long nd = (long long)H.n * nL, nf = (long long)H.n * H.r;
    LSW_TRY(pool_alloc(reinterpret_cast<void**>(&B.D), sizeof(uint32_t) * nd));
    B.bytes = sizeof(uint32_t) * nd;
    k_to_bf16<<<gridn(nd), 256, 0, st>>>(H.D, B.D, nd);
    LSW_LAUNCH_CHECK();
    B.U.assign(H.L + 1, nullptr);
    B.W.assign(H.L + 1, nullptr);
    B.ulay.assign(H.L + 1, FAC_PLAIN);
    B.wlay.assign(H.L + 1, FAC_PLAIN);
    // levels whose blocks the tensor-core kernels take are stored as their
    // operand tiles: W for the partials W^H x, U for the products U t
    B.rp = (H.r + 7) & ~7;
    for (int l = 1; l <= H.L; ++l) {
        const int nb = H.nl(l);
        const bool tiled = nb % 128 == 0 && B.rp <= 64;
        const long long nfl = tiled ? (long long)H.n * B.rp : nf;
        LSW_TRY(pool_alloc(reinterpret_cast<void**>(&B.U[l]), sizeof(uint32_t) * nfl));
        LSW_TRY(pool_alloc(reinterpret_cast<void**>(&B.W[l]), sizeof(uint32_t) * nfl));
        B.bytes += 2 * sizeof(uint32_t) * nfl;
        if (tiled) {
            B.ulay[l] = FAC_TILE_A;
            B.wlay[l] = FAC_TILE_P;
            k_to_bf16_fac<<<gridn(nfl), 256, 0, st>>>(H.U[l], B.U[l], FAC_TILE_A, nb, H.r, B.rp, H.n / nb);
            LSW_LAUNCH_CHECK();
            k_to_bf16_fac<<<gridn(nfl), 256, 0, st>>>(H.W[l], B.W[l], FAC_TILE_P, nb, H.r, B.rp, H.n / nb);
            LSW_LAUNCH_CHECK();
        } else {
            k_to_bf16<<<gridn(nf), 256, 0, st>>>(H.U[l], B.U[l], nf);
            LSW_LAUNCH_CHECK();
            k_to_bf16<<<gridn(nf), 256, 0, st>>>(H.W[l], B.W[l], nf);
            LSW_LAUNCH_CHECK();
        }
    }
    LSW_CUDA(cudaStreamSynchronize(st));
    return LSW_OK;
}

// Y = H X for the whole matrix on BF16 storage (tree order, k columns, ld n)
lsw_status hmv_bf16(const HStoreB& B, const float2* X, int k, float2* Y, cudaStream_t st) {
    const int n = B.n, L = B.L, r = B.r, nL = B.nl(L), nleaf = 1 << L;
    for (int c0 = 0; c0 < k; c0 += 32) {
        const int kc = std::min(32, k - c0);
        if (tc_gemm_enabled() && tc_bf16_fits(nL, kc, nL)) {
            LSW_TRY(cgemm_tc_bf16(B.D, nL, (long long)nL * nL, X + (size_t)c0 * n, n, nL, Y + (size_t)c0 * n, n, nL, nL,
                                  kc, nL, make_float2(1.f, 0.f), nleaf, st));
        } else {
            k_leaf_bf16<<<gridn((long long)n * kc), 256, 0, st>>>(B.D, X + (size_t)c0 * n, Y + (size_t)c0 * n, nL,
                                                                 nleaf, kc, n);
            LSW_LAUNCH_CHECK();
        }
    }
    if (L < 1) return LSW_OK;
    if ((nL & 3) || L > kMaxLev || r > 64) return LSW_ERR_UNSUPPORTED_SIZE;
    // every level's U (W^H x[sibling]) in column blocks the fused kernels take
    const int kb = std::max(1, std::min(64, 4096 / r));
    for (int c0 = 0; c0 < k; c0 += kb) {
        const int kc = std::min(kb, k - c0);
        LrLevels<float2, uint32_t> lv;
        lv.nlev = L;
        lv.rp = B.rp;
        lv.chunk0[0] = 0;
        lv.t0[0] = 0;
        for (int q = 0; q < L; ++q) {
            const int lp = 1 + q, cnt = 1 << lp, nb = B.nl(lp);
            lv.F[q] = B.W[lp];
            lv.G[q] = B.U[lp];
            lv.flay[q] = B.wlay[lp];
            lv.glay[q] = B.ulay[lp];
            lv.nb[q] = nb;
            lv.ch[q] = std::min(nb, 2048);
            lv.chunk0[q + 1] = lv.chunk0[q] + n / lv.ch[q];
            lv.t0[q + 1] = lv.t0[q] + cnt;
        }
        for (int q = L; q < kMaxLev; ++q) {
            lv.F[q] = lv.G[q] = nullptr;
            lv.nb[q] = lv.ch[q] = 1;
            lv.chunk0[q + 1] = lv.chunk0[q];
            lv.t0[q + 1] = lv.t0[q];
        }
        LSW_TRY((lr_launch<float2, uint32_t>(lv, n, r, kc, X + (size_t)c0 * n, Y + (size_t)c0 * n, 1, 0, st)));
    }
    return LSW_OK;
}

// y = H x (grid order, nb fields)
template <typename R>
lsw_status apply_h(const lsw_hmatrix* h, const typename Cx<R>::T* x, typename Cx<R>::T* y, int nb, cudaStream_t st) {
    typedef typename Cx<R>::T C;
    const int n = h->n, r = h->r;
    if (nb <= 0) return LSW_OK;
    if (h->kind == LSW_H_LOWRANK_SMW) {
        const C* U = (const C*)h->smwU;
        const C* W = (const C*)h->smwW;
        const C* Z = (const C*)h->smwZ;
        DevBuf t1, t2;
        LSW_TRY(t1.alloc(sizeof(C) * (size_t)r * nb, st));
        LSW_TRY(t2.alloc(sizeof(C) * (size_t)r * nb, st));
        // y = x + U (Z (W^H x))   (Eq. 12 applied as three factors, Eq. 14)
        LSW_TRY(gemm<R>('C', 'N', r, nb, n, one<C>(), W, n, 0, x, n, 0, zero<C>(), t1.as<C>(), r, 0, 1, st));
        LSW_TRY(gemm<R>('N', 'N', r, nb, r, one<C>(), Z, r, 0, t1.as<C>(), r, 0, zero<C>(), t2.as<C>(), r, 0, 1, st));
        LSW_CUDA(cudaMemcpyAsync(y, x, sizeof(C) * (size_t)n * nb, cudaMemcpyDeviceToDevice, st));
        LSW_TRY(gemm<R>('N', 'N', n, nb, r, one<C>(), U, n, 0, t2.as<C>(), r, 0, one<C>(), y, n, 0, 1, st));
        return LSW_OK;
    }
    if (sizeof(R) == 4 && h->bf16) {
        DevBuf xt, yt;
        LSW_TRY(xt.alloc(sizeof(C) * (size_t)n * nb, st));
        LSW_TRY(yt.alloc(sizeof(C) * (size_t)n * nb, st));
        k_permute<C><<<gridn((long long)n * nb), 256, 0, st>>>(x, xt.as<C>(), h->perm_d, n, nb, 0);
        LSW_LAUNCH_CHECK();
        LSW_TRY(hmv_bf16(h->hb, reinterpret_cast<const float2*>(xt.p), nb, reinterpret_cast<float2*>(yt.p), st));
        k_permute<C><<<gridn((long long)n * nb), 256, 0, st>>>(yt.as<C>(), y, h->perm_d, n, nb, 1);
        LSW_LAUNCH_CHECK();
        return LSW_OK;
    }
    const HStore<R>& H = *reinterpret_cast<const HStore<R>*>(sizeof(R) == 8 ? (const void*)&h->h64 : (const void*)&h->h32);
    DevBuf xt, yt, T;
    LSW_TRY(xt.alloc(sizeof(C) * (size_t)n * nb, st));
    LSW_TRY(yt.alloc(sizeof(C) * (size_t)n * nb, st));
    LSW_TRY(T.alloc(sizeof(C) * ((size_t)1 << h->L) * r * nb, st));
    k_permute<C><<<gridn((long long)n * nb), 256, 0, st>>>(x, xt.as<C>(), h->perm_d, n, nb, 0);
    LSW_LAUNCH_CHECK();
    LSW_TRY(hmv<R>(H, 0, 0, xt.as<C>(), nb, yt.as<C>(), T.as<C>(), st));
    k_permute<C><<<gridn((long long)n * nb), 256, 0, st>>>(yt.as<C>(), y, h->perm_d, n, nb, 1);
    LSW_LAUNCH_CHECK();
    return LSW_OK;
}

int hmatrix_prec(const lsw_hmatrix* h) { return h->prec; }

template lsw_status apply_h<float>(const lsw_hmatrix*, const float2*, float2*, int, cudaStream_t);
template lsw_status apply_h<double>(const lsw_hmatrix*, const double2*, double2*, int, cudaStream_t);

}  // namespace lsw

using namespace lsw;

extern "C" {

lsw_status lsw_sketch_range(const lsw_green* g, int prec, const double* chi, lsw_box rows, lsw_box cols, int rank,
                            int oversample, int q, uint64_t seed, uint32_t stream_id, void* U, void* W, void* stream) {
    if (!g || !chi || !U || !W || rank <= 0 || oversample < 0 || q < 0) return LSW_ERR_INVALID_ARG;
    if (rank + oversample > 64) return LSW_ERR_INVALID_ARG;
    auto inside = [&](lsw_box b) {
        return b.z0 >= 0 && b.z1 <= g->nz && b.x0 >= 0 && b.x1 <= g->nx && b.z0 < b.z1 && b.x0 < b.x1;
    };
    if (!inside(rows) || !inside(cols)) return LSW_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const uint32_t w2 = stream_w2(TAG_GLOBAL, 0, 0, 0);
    if (prec == LSW_C128)
        return sketch_boxes<double>(g, chi, rows, cols, rank, oversample, q, seed, w2, stream_id, one<double2>(),
                                    (double2*)U, (double2*)W, st);
    if (prec == LSW_C64)
        return sketch_boxes<float>(g, chi, rows, cols, rank, oversample, q, seed, w2, stream_id, one<float2>(),
                                   (float2*)U, (float2*)W, st);
    return LSW_ERR_INVALID_ARG;
}

lsw_status lsw_build_hmatrix(const lsw_green* g, const double* chi, const lsw_hparams* hp, void* stream,
                             lsw_hmatrix** out) {
    if (!g || !chi || !hp || !out) return LSW_ERR_INVALID_ARG;
    *out = nullptr;
    if (hp->prec != LSW_C128 && hp->prec != LSW_C64 && !(hp->prec == LSW_BF16 && hp->kind == LSW_H_HODLR))
        return LSW_ERR_INVALID_ARG;
    if (hp->rank <= 0 || hp->oversample < 0 || hp->q < 0 || hp->rank + hp->oversample > 64) return LSW_ERR_INVALID_ARG;
    if (hp->kind != LSW_H_LOWRANK_SMW && hp->kind != LSW_H_HODLR) return LSW_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    lsw_hmatrix* h = new (std::nothrow) lsw_hmatrix();
    if (!h) return LSW_ERR_OOM;
    h->kind = hp->kind;
    h->prec = hp->prec == LSW_BF16 ? LSW_C64 : hp->prec;     // vectors are complex64 for BF16 storage
    h->n = g->nz * g->nx;
    h->nz = g->nz;
    h->nx = g->nx;
    h->r = hp->rank;
    lsw_status s = LSW_OK;
    if (hp->kind == LSW_H_LOWRANK_SMW) {
        s = hp->prec == LSW_C128 ? build_smw<double>(g, chi, hp, h, st) : build_smw<float>(g, chi, hp, h, st);
    } else {
        if (hp->levels < 1 || hp->levels > 12 || (hp->split != LSW_SPLIT_QUADTREE && hp->split != LSW_SPLIT_STRIPS)) {
            delete h;
            return LSW_ERR_INVALID_ARG;
        }
        h->L = hp->levels;
        s = h->tree.init(g->nz, g->nx, hp->levels, hp->split);
        if (s == LSW_OK) {
            const size_t pb = sizeof(int) * h->tree.perm.size();
            if (cudaMalloc(&h->perm_d, pb) != cudaSuccess) s = LSW_ERR_OOM;
            else if (cudaMemcpy(h->perm_d, h->tree.perm.data(), pb, cudaMemcpyHostToDevice) != cudaSuccess) s = LSW_ERR_CUDA;
        }
        if (s == LSW_OK) {
            if (hp->prec == LSW_C128) {
                s = build_hodlr<double>(g, chi, hp, h, st, h->h64);
                h->bytes = h->h64.bytes;
            } else {
                s = build_hodlr<float>(g, chi, hp, h, st, h->h32);
                h->bytes = h->h32.bytes;
                if (s == LSW_OK && hp->prec == LSW_BF16) {
                    s = to_bf16(h->h32, h->hb, st);
                    if (s == LSW_OK) {
                        h->h32.release();
                        h->bf16 = true;
                        h->bytes = h->hb.bytes;
                    }
                }
            }
        }
    }
    if (s != LSW_OK) {
        lsw_destroy_hmatrix(h);
        return s;
    }
    *out = h;
    return LSW_OK;
}

lsw_status lsw_destroy_hmatrix(lsw_hmatrix* h) {
    if (!h) return LSW_ERR_INVALID_ARG;
    h->h32.release();
    h->h64.release();
    h->hb.release();
    if (h->perm_d) cudaFree(h->perm_d);
    if (h->smwU) cudaFree(h->smwU);
    if (h->smwW) cudaFree(h->smwW);
    if (h->smwZ) cudaFree(h->smwZ);
    delete h;
    return LSW_OK;
}

lsw_status lsw_hmatrix_bytes(const lsw_hmatrix* h, uint64_t* bytes) {
    if (!h || !bytes) return LSW_ERR_INVALID_ARG;
    *bytes = h->bytes + sizeof(int) * (size_t)h->n * (h->perm_d ? 1 : 0);
    return LSW_OK;
}

lsw_status lsw_apply_precond(const lsw_hmatrix* h, const void* x, void* y, int nbatch, void* stream) {
    if (!h || nbatch < 0) return LSW_ERR_INVALID_ARG;
    if (nbatch == 0) return LSW_OK;
    if (!x || !y || x == y) return LSW_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (h->prec == LSW_C128) return apply_h<double>(h, (const double2*)x, (double2*)y, nbatch, st);
    return apply_h<float>(h, (const float2*)x, (float2*)y, nbatch, st);
}

}  // extern "C"
