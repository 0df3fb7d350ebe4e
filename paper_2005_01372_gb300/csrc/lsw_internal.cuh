// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>
#include <vector>

#include "lsw.h"

namespace lsw {

// ------------------------------------------------------------ complex types
template <typename R> struct Cx;
template <> struct Cx<float>  { typedef float2 T; };
template <> struct Cx<double> { typedef double2 T; };

__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }

template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { return mk(a.x + b.x, a.y + b.y); }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { return mk(a.x - b.x, a.y - b.y); }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
template <typename C> __host__ __device__ __forceinline__ C cmulc(C a, C b) {
    return mk(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { return mk(a.x, -a.y); }
template <typename C, typename R> __host__ __device__ __forceinline__ C cscale(C a, R s) { return mk(a.x * s, a.y * s); }
template <typename C> __host__ __device__ __forceinline__ C czero() { C z; z.x = 0; z.y = 0; return z; }
// acc += a * b
template <typename C> __device__ __forceinline__ void cfma(C& acc, C a, C b) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <typename C> __device__ __forceinline__ void cfmac(C& acc, C a, C b) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
}

// ------------------------------------------------------------------ errors
#define LSW_CUDA(call)                                             \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) {                                   \
            lsw::set_last_error(e_, #call, __FILE__, __LINE__);    \
            return e_ == cudaErrorMemoryAllocation ? LSW_ERR_OOM : LSW_ERR_CUDA; \
        }                                                          \
    } while (0)
#define LSW_TRY(expr)                                              \
    do {                                                           \
        lsw_status s_ = (expr);                                    \
        if (s_ != LSW_OK) return s_;                               \
    } while (0)
// Every kernel launch of the library is followed by exactly one
// LSW_LAUNCH_CHECK(), which also counts it (lsw_launch_count()).
#define LSW_LAUNCH_CHECK()            \
    do {                              \
        lsw::count_launch();          \
        LSW_CUDA(cudaGetLastError()); \
    } while (0)

void set_last_error(cudaError_t e, const char* what, const char* file, int line);
void count_launch();
// Add n launches to the counter (the kernels of a CUDA graph replay; n < 0
// takes back kernels that were captured but never ran).
void count_launches(long long n);
unsigned long long launch_counter();
void count_graph_replay();
// Process-wide switch (default on) for replaying captured CUDA graphs.
bool graphs_enabled();

// Diagnostic timing of one kernel family (lsw_kernel_timer_*): while the
// family named at lsw_kernel_timer_start is enabled, a KTimer records CUDA
// events on the launching stream around the launches it scopes and adds the
// algorithmic bytes and flops its caller states.
// Work captured into a CUDA graph is timed too: the events are recorded as
// nodes of the graph, the owner of the graph takes them with
// timer_take_captured() when the capture ends and adds each replay's elapsed
// times with timer_harvest() once the replay has finished.
class KTimer {
  public:
    KTimer(const char* family, cudaStream_t st, double bytes, double flops);
    ~KTimer();

  private:
    cudaEvent_t e0_ = nullptr, e1_ = nullptr;
    cudaStream_t st_ = nullptr;
    double bytes_ = 0, flops_ = 0;
    bool captured_ = false;
};
struct TimedSpan {
    cudaEvent_t e0, e1;
    double bytes, flops;
};
std::vector<TimedSpan> timer_take_captured();
void timer_harvest(const std::vector<TimedSpan>& spans);
void timer_release(std::vector<TimedSpan>& spans);

inline bool is_pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }
inline int ilog2(long long v) { int l = 0; while ((1LL << l) < v) ++l; return l; }

// Stream-ordered scratch that frees itself.
struct DevBuf {
    void* p = nullptr;
    cudaStream_t s = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { if (p) cudaFreeAsync(p, s); }
    lsw_status alloc(size_t bytes, cudaStream_t st) {
        if (p) { cudaFreeAsync(p, s); p = nullptr; }
        s = st;
        if (bytes == 0) bytes = 16;
        cudaError_t e = cudaMallocAsync(&p, bytes, st);
        if (e != cudaSuccess) { p = nullptr; set_last_error(e, "cudaMallocAsync", __FILE__, __LINE__);
                                return e == cudaErrorMemoryAllocation ? LSW_ERR_OOM : LSW_ERR_CUDA; }
        return LSW_OK;
    }
    template <typename T> T* as() const { return static_cast<T*>(p); }
};

// Fork independent work from a parent stream onto library-owned streams and
// join it back: child(i) starts after everything enqueued on the parent so
// far; join() makes the parent wait for every child used.
// Host worker threads of a batched call fork onto their own stream pools.
void set_worker_slot(int slot);

class Fork {
  public:
    explicit Fork(cudaStream_t parent);
    ~Fork();
    cudaStream_t child(int i);
    lsw_status join();

  private:
    cudaStream_t parent_;
    cudaEvent_t start_ = nullptr;
    unsigned used_ = 0;
    cudaStream_t streams_[8] = {};
};

// ------------------------------------------------------------ FFT geometry
// One spectrum of a (bz x bx) box: the FFT of the even extension of the
// Green table to (2bz x 2bx), scaled by 1/(4 bz bx), as its quarter
// (bx + 1) x (bz + 1), kx-major.
struct Spectrum {
    int bz = 0, bx = 0;
    double2* q64 = nullptr;
    float2* q32 = nullptr;
    double2* t64 = nullptr;   // the same quarter, kz-major: (bz + 1) x (bx + 1)
    float2* t32 = nullptr;
};

}  // namespace lsw

struct lsw_green {
    int device;
    int nz, nx;
    double h, c0, freq, k;
    double2* table = nullptr;            // (nx+1) x (nz+1), entry dx*(nz+1)+dz
    lsw::Spectrum full;                  // spectrum of the whole grid
    int twP = 0;                         // twiddle table length (max FFT size)
    double2* tw64 = nullptr;             // tw[m] = exp(-2 pi i m / twP)
    float2* tw32 = nullptr;
};

namespace lsw {

// ---------------------------------------------------- operator (fft_op.cu)
// Geometry of one batched operator launch on boxes of extent (bz, bx):
// vector b lives at base + b * vstride, its box origin is origin[b / vpb]
// (NULL: the grid origin), chi is read at chi[(x0 + ix) * chi_ld + z0 + iz].
struct OpGeom {
    int bz, bx;
    const double* chi;
    int chi_ld;
    const int2* origin;   // device, may be NULL
    int vpb;              // vectors per box
};

template <typename R>
lsw_status op_apply(const lsw_green* g, const Spectrum& sp, const OpGeom& geo, int mode,
                    const typename Cx<R>::T* u, const typename Cx<R>::T* u0, typename Cx<R>::T* y,
                    int nbatch, typename Cx<R>::T* work, cudaStream_t st);

lsw_status build_spectrum(const lsw_green* g, int bz, int bx, Spectrum* out, cudaStream_t st);
void free_spectrum(Spectrum* s);

// ------------------------------------------------------ dense helpers (la.cu)
// Batched complex GEMM, column-major:  C_b = alpha * op(A_b) * op(B_b) + beta * C_b
// op: 'N' or 'C' (conjugate transpose).  A_b = A + b * sA, etc.
template <typename R>
lsw_status gemm(char opA, char opB, int m, int n, int k, typename Cx<R>::T alpha,
                const typename Cx<R>::T* A, int lda, long long sA,
                const typename Cx<R>::T* B, int ldb, long long sB,
                typename Cx<R>::T beta, typename Cx<R>::T* C, int ldc, long long sC,
                int batch, cudaStream_t st);

// Batched thin Householder QR: A_b (m x k, ld m) is replaced by Q_b with
// orthonormal columns spanning range(A_b) (k <= 64, m >= 1).
template <typename R>
lsw_status qr_explicit(typename Cx<R>::T* A, int m, int k, long long sA, int batch,
                       typename Cx<R>::T* work, cudaStream_t st);

// Batched Gram matrices G_b = Y_b^H Y_b (k x k, k <= 64) accumulated in FP64.
template <typename R>
lsw_status gram64(const typename Cx<R>::T* Y, int m, int k, long long sY, int batch,
                  double2* G, cudaStream_t st);

// Batched Hermitian eigenvectors by cyclic Jacobi in precision R: V_b (k x k)
// receives the eigenvectors of the FP64 matrix G_b as columns, sorted by
// decreasing eigenvalue.  polish 1: for a nearly diagonal G whose small
// eigenvalues are to be resolved relative to themselves (no global stop on
// the off-diagonal norm, a tighter pair threshold); polish 2: a coarse first
// pass (stop at a relative squared off-diagonal norm of 1e-6) for a polish
// run to finish.
template <typename R>
lsw_status heev_jacobi(const double2* G, typename Cx<R>::T* V, int k, int batch, cudaStream_t st, int polish = 0);

// FP64 small-matrix arithmetic of the sketches (small64.cu).
// Gram matrices of complex64 blocks with error-free products (Dot2), FP64 result.
// Blocks b with active[b] == 0 are skipped (active may be NULL: all).
lsw_status gram64_c64(const float2* Y, int m, int k, long long sY, int batch, double2* G, cudaStream_t st,
                      const int* active = nullptr);
// Rinv_b = R_b^-1 (upper triangular, k x k) with G_b + s I = R_b^H R_b, an
// FP64 Cholesky factor, s = shift_rel tr(G_b) / k (raised on breakdown).
// active (may be NULL) skips blocks; need2 (may be NULL) receives 1 where a
// second Cholesky QR pass is needed (kappa_F > 1e3 or a shift was applied).
template <typename R>
lsw_status chol_rinv(const double2* G, int k, int batch, double shift_rel, typename Cx<R>::T* Rinv, cudaStream_t st,
                     const int* active = nullptr, int* need2 = nullptr);
// Eigenvectors of the FP64 Hermitian G_b as the columns of V_b (k x k, FP32),
// by decreasing eigenvalue, resolved to FP64 accuracy: a coarse FP32 Jacobi
// (V0), an FP64-accurate Rayleigh-Ritz projection B = V0^H G V0, FP32 Jacobi
// on the nearly diagonal B, V = V0 Z.
lsw_status heev_c64(const double2* G, float2* V, int k, int batch, cudaStream_t st);
// Thin QR of complex64 sketch blocks (Q in place): Cholesky QR with Dot2
// Grams and products and FP64 factors, a second pass where the conditioning
// asks for it; FP64 Householder for short blocks.
lsw_status qr_sketch_c64(float2* A, int m, int k, long long sA, int batch, cudaStream_t st);

// Cast FP64 complex -> working precision.
template <typename R>
lsw_status cast_from64(const double2* src, typename Cx<R>::T* dst, long long n, cudaStream_t st);

// Philox4x32-10 complex Gaussian probe blocks: block b (m x k, ld m) at
// dst + b * sD uses stream words w2[b], w3[b] (device arrays).
template <typename R>
lsw_status gaussian_fill(typename Cx<R>::T* dst, int m, int k, long long sD, int batch,
                         uint64_t seed, const uint32_t* w2, const uint32_t* w3, cudaStream_t st);

// Batched in-place inverse of n x n matrices (Gauss-Jordan, partial pivoting).
template <typename R>
lsw_status inverse_gj(typename Cx<R>::T* A, int n, long long sA, int batch, cudaStream_t st);

// Batched complex FP32 GEMM C_b = alpha A_b B_b on the tcgen05 tensor cores
// (3xTF32, FP32 accuracy), column-major, for M % 128 == 0, K % 16 == 0,
// 1 <= N <= 32 (tc_gemm.cu).  tc_gemm_enabled: the process-wide switch.
bool tc_gemm_enabled();
void tc_gemm_enable(bool on);
bool tc_gemm_fits(int M, int N, int K);
lsw_status cgemm_tc(const float2* A, int lda, long long sA, const float2* B, int ldb, long long sB, float2* C, int ldc,
                    long long sC, int M, int N, int K, float2 alpha, int batch, cudaStream_t st);
// The same with A stored as BF16 (re, im) pairs, one 32-bit word per entry
// (kind::f16 MMAs, B split into BF16 hi + lo): M % 128 == 0, K % 32 == 0.
bool tc_bf16_fits(int M, int N, int K);
lsw_status cgemm_tc_bf16(const uint32_t* A, int lda, long long sA, const float2* B, int ldb, long long sB, float2* C,
                         int ldc, long long sC, int M, int N, int K, float2 alpha, int batch, cudaStream_t st);

// ------------------------------------------- H-matrix level products
// Every level of a subtree product at once: level q has blocks of nb[q] rows
// whose factors F_j, G_j (nb x r, column-major) are consecutive; rows are cut
// into chunks of ch[q] for the partial products (hmatrix.cu, lr_tc.cu).
constexpr int kMaxLev = 16;
template <typename C, typename FT = C> struct LrLevels {
    const FT* F[kMaxLev];
    const FT* G[kMaxLev];
    int nb[kMaxLev];
    int ch[kMaxLev];                // rows per chunk (divides nb)
    int chunk0[kMaxLev + 1];        // first chunk of each level
    long long t0[kMaxLev + 1];      // first T block of each level (units of r*k)
    int nlev;
    int flay[kMaxLev] = {};         // storage of F and G per level (FAC_*)
    int glay[kMaxLev] = {};
    int rp = 0;                     // columns per block of the tiled storages
};

// Storage of a level's factor (a block of nb rows and r columns):
//   FAC_PLAIN: column-major, block after block (nb * r entries each);
//   FAC_TILE_P: the operand tiles of the partial products F^H x: per block,
//     per group of 8 rows, the rp columns (r rounded up to 8, zero-padded)
//     as 8-column x 16-byte core matrices (4 rows of complex per 16 bytes);
//   FAC_TILE_A: the operand tiles of the products G t: per block, per tile
//     of 128 rows, per group of 8 columns, the 128 rows as 8-row x 16-byte
//     core matrices (4 columns of complex per 16 bytes).
// Either tile is the canonical K-major, non-swizzled tensor-core layout of a
// 16-element BF16 K-step (two core matrices 128 B apart along K, 8-row
// groups 256 B apart), so a stage of the tensor-core kernels is one
// contiguous copy.
enum { FAC_PLAIN = 0, FAC_TILE_P = 1, FAC_TILE_A = 2 };
__host__ __device__ __forceinline__ long long fac_index(int lay, int nb, int r, int rp, int j, int o, int i) {
    if (lay == FAC_PLAIN) return ((long long)j * r + i) * nb + o;
    const long long base = (long long)j * nb * rp;
    if (lay == FAC_TILE_P)
        return base + (long long)(o >> 3) * (rp * 8) + (i >> 3) * 64 + ((o & 7) >> 2) * 32 + (i & 7) * 4 + (o & 3);
    return base + ((long long)(o >> 7) * (rp >> 3) + (i >> 3)) * 1024 + ((o & 127) >> 3) * 64 + ((i & 7) >> 2) * 32 +
           (o & 7) * 4 + (i & 3);
}
// tcgen05 forms for BF16 factors (lr_tc.cu): the partials P = F^H X per
// chunk, and Y += sum over levels of G T.
bool lr_tc_fits(const LrLevels<float2, uint32_t>& lv, int m, int r, int k);
lsw_status lr_partial_tc(const LrLevels<float2, uint32_t>& lv, int m, int r, int k, const float2* X, int swapA,
                         float2* P, cudaStream_t st);
lsw_status lr_apply_tc(const LrLevels<float2, uint32_t>& lv, int m, int r, int k, const float2* T, int swapC,
                       float2* Y, cudaStream_t st);

// Per-field FP64 squared 2-norms: out[b] = sum |x_b|^2 over n entries.
template <typename R>
lsw_status norms2(const typename Cx<R>::T* x, long long n, int batch, double* out, cudaStream_t st);

}  // namespace lsw
