// Launchers of the hot-path sparse kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace nm {

// Process-wide count of kernels launched by the library (nm_kernel_launches).
void count_launch(uint64_t n = 1);
uint64_t launches_so_far();

enum KronMode { KRON_PLAIN = 0, KRON_CHEB = 1, KRON_CHEB_FILT = 2, KRON_CORI = 3 };

// Row tiles of a scalar CSR matrix for the bulk-copy staged mass step
// (mass_tma.cu): tile t covers rows [r0, r1) (at most kTmaRows rows, at
// most kTmaDcap distinct neighbour nodes, at most kTmaEcap stored
// entries); its distinct neighbour nodes are ucol[u0 .. u0 + nu) and
// lcol[e] is the position of entry e's column in that list. vals, rowptr,
// dinv are padded copies of the float matrix (so that 16-byte windows
// never leave the allocation); ldiag[i] is the position of row i's own
// node in its tile's list. err: a device flag a timed-out wait sets.
constexpr int kTmaRows = 32;
constexpr int kTmaDcap = 160;
constexpr int kTmaEcap = 1024;
struct TmaTiles {
    int ntiles = 0;
    const int4* desc = nullptr;     // (r0, r1, u0, nu) per tile
    const int* ucol = nullptr;
    const uint16_t* lcol = nullptr;
    const float* vals = nullptr;
    const int* rowptr = nullptr;
    const float* dinv = nullptr;
    const uint16_t* ldiag = nullptr;
    int* err = nullptr;
};

// Y (or the Chebyshev / filter epilogue) from the scalar CSR matrix A
// applied as A (x) I_R to row-major blocks of b columns. A node row i owns
// the R consecutive rows R*i .. R*i+R-1 of every block.
template <typename T>
struct KronArgs {
    int nrows = 0;
    const int* rowptr = nullptr;
    const int* col = nullptr;
    const T* val = nullptr;
    const T* dinv = nullptr;
    int b = 0;
    const T* X = nullptr;   int64_t ldx = 0;   // gathered operand x_k
    T* Y = nullptr;         int64_t ldy = 0;   // PLAIN / CORI output
    const T* W = nullptr;   int64_t ldw = 0;   // CHEB right-hand side
    const T* Xp = nullptr;  int64_t ldp = 0;   // CHEB x_{k-1} (nullptr: zero)
    T* Xn = nullptr;        int64_t ldn = 0;   // CHEB x_{k+1} (may alias Xp)
    T om = 0, inv_theta = 0;
    const T* Tk = nullptr;  int64_t ldtk = 0;  // FILT current Chebyshev block
    const T* Tp = nullptr;  int64_t ldtp = 0;  // FILT previous (nullptr: zero)
    T* Tn = nullptr;        int64_t ldtn = 0;  // FILT next (may alias Tp)
    T* Z = nullptr;         int64_t ldz = 0;   // FILT accumulator (nullptr: none)
    T a1 = 0, cshift = 0, a2 = 0, gam = 0;
    const double* gam_tab = nullptr;   // FILT: per column group gamma (overrides gam)
    int gam_group = 1;                 // columns per group
    T sk[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};      // CORI 3x3 (row-major)
    // optional row tiles (see DevCSR): float operands with b = 32 and
    // ldx = 32 then gather through shared memory
    const int* tile_uptr = nullptr;
    const int* tile_ucol = nullptr;
    const uint16_t* lcol = nullptr;
    int tile_rows = 0;
    int64_t ntiles = 0;
    int tile_umax = 0;
    int tile_kernel = 2;   // 1: 256-thread rounds, 2: 512-thread unrolled rounds
    // SM-local persistent schedule (b = 32 or 64): nreg region counters,
    // zeroed by the launcher on the stream before the launch
    int* sched = nullptr;
    int nreg = 0;
    // chunked warp-per-row schedule (b = 17..64): threads per CTA
    // (256, 512 or 1024), 0 = off
    int chunk = 0;
    // float blocks 32 wide with ldx = 32: 1 = 16-byte vectorised gathers
    // (four groups of eight lanes per row), 0 = scalar gathers
    int vec = 1;
    int vec_threads = 32;    // CTA size of the vectorised kernel, R = 3 (32 .. 1024, power of two)
    int vec_threads_p = 128; // the same for R = 1
    // bulk-copy staged tiles (R = 3, float, b = ldx = 32, CHEB): ntiles > 0 selects mass_tma.cu
    TmaTiles tma;
};

// The staged float mass step (one Chebyshev semi-iteration step of
// M_rho (x) I_3 on 32 columns): persistent CTAs, one producer warp filling
// two shared-memory stages by cp.async.bulk, eight consumer warps.
int launch_kron_tma(const KronArgs<float>& a, cudaStream_t s);
// Host check of the device flag of a staged kernel (synchronises stream s):
// NM_OK, or NM_ETIMEOUT if a bounded wait of a launch ran out.
int tma_status(int* err_dev, cudaStream_t s);

template <typename T>
int launch_kron(int R, int mode, const KronArgs<T>& a, cudaStream_t s);

// W = A X (+ E S) for the 3x3-block CSR A over u-nodes and the optional
// 3x1-block CSR E (u-nodes x p-nodes) applied to the pressure block S.
// With X1 != nullptr also writes the first semi-iterate X1 = inv_theta *
// dinv[i] * W of the mass solve.
template <typename T>
struct Bsr33Args {
    int nrows = 0;
    const int* rowptr = nullptr;
    const int* col = nullptr;
    const T* val = nullptr;
    const int* e_rowptr = nullptr;
    const int* e_col = nullptr;
    const T* e_val = nullptr;
    const T* S = nullptr;   int64_t lds = 0;
    int b = 0;
    const T* X = nullptr;   int64_t ldx = 0;
    T* W = nullptr;         int64_t ldw = 0;
    T* X1 = nullptr;        int64_t ldx1 = 0;
    const T* dinv = nullptr;
    T inv_theta = 0;
};

template <typename T>
int launch_bsr33(const Bsr33Args<T>& a, cudaStream_t s);

// Q = E^T X for the 1x3-block CSR E^T (p-nodes x u-nodes); with S1 !=
// nullptr also S1 = inv_theta * dinv[p] * Q.
template <typename T>
struct Bsr13Args {
    int nrows = 0;
    const int* rowptr = nullptr;
    const int* col = nullptr;
    const T* val = nullptr;
    int b = 0;
    const T* X = nullptr;   int64_t ldx = 0;
    T* Q = nullptr;         int64_t ldq = 0;
    T* S1 = nullptr;        int64_t lds1 = 0;
    const T* dinv = nullptr;
    T inv_theta = 0;
};

template <typename T>
int launch_bsr13(const Bsr13Args<T>& a, cudaStream_t s);

// X[(R i + k), c] = inv_theta * dinv[i] * W[(R i + k), c] (first semi-iterate).
template <typename T>
int launch_dscale(int R, int64_t nodes, int b, T inv_theta, const T* dinv, const T* W, int64_t ldw, T* X,
                  int64_t ldx, cudaStream_t s);

// r32 = float(W - (A (x) I_R) x32) with double matrix values and double
// sums over the float iterate (the refinement residual of a mixed solve).
int launch_resid_mixed(int R, int64_t nodes, const int* rowptr, const int* col, const double* val,
                       const double* W, int64_t ldw, const float* x32, float* r32, int b, cudaStream_t s);

// S = double(x32) + double(e32); with Tn != nullptr the outer filter update
// Tn = a1 (S - c Tk) - a2 Tp, Z += gam Tn, else out = S.
struct CombineArgs {
    int64_t rows = 0;
    int b = 0;
    const float* x32 = nullptr;
    const float* e32 = nullptr;
    double* out = nullptr;
    const double* Tk = nullptr;
    const double* Tp = nullptr;
    double* Tn = nullptr;
    double* Z = nullptr;
    int64_t ldz = 0;
    double a1 = 0, cshift = 0, a2 = 0, gam = 0;
    const double* gam_tab = nullptr;   // per column group gamma (overrides gam)
    int gam_group = 1;
    float* Th = nullptr;   // optional exact float pair (hi, lo) of Tn, dense
    float* Tl = nullptr;
    // graph replay: gamma = gam_tab[(deg[0] + 1) * gam_stride + c / gam_group]
    // with the degree read from device memory (overrides gam and gam_tab's
    // host-side offset)
    const int* deg = nullptr;
    int gam_stride = 0;
};
int launch_combine(const CombineArgs& a, cudaStream_t s);
// One-thread kernels that set / advance the device-side degree counter of
// a replayed filter graph.
int launch_set_int(int* p, int v, cudaStream_t s);
int launch_inc_int(int* p, cudaStream_t s);
// W[3i + m, c] += sum_f E[f, m] S[col(f), c]: the fluid coupling term of
// K_eff added to a finished A_G product (3x1-block CSR over u-node rows).
int launch_bsr31_add(int nrows, const int* rowptr, const int* col, const double* val, const double* S, int64_t lds,
                     int b, double* W, int64_t ldw, cudaStream_t s);

// Double-float forms (value = hi + lo, two floats, ~2^-48 relative): the
// K_eff SpMM and the refinement residual on the float units.
// Split a double block into exact float pairs (hi = fl(x), lo = fl(x - hi)).
int launch_split(int64_t rows, int b, const double* X, int64_t ldx, float* Xh, float* Xl, cudaStream_t s);
// W = A X + E S with A's 3x3 blocks as (hi, lo) floats and X as (hi, lo)
// float blocks (ld b), double-float sums; the optional E S part in double.
struct Bsr33DfArgs {
    int nrows = 0;
    const int* rowptr = nullptr;
    const int* col = nullptr;
    const float* vh = nullptr;
    const float* vl = nullptr;
    const float* Xh = nullptr;
    const float* Xl = nullptr;
    int b = 0;
    const int* e_rowptr = nullptr;
    const int* e_col = nullptr;
    const double* e_val = nullptr;
    const double* S = nullptr;
    int64_t lds = 0;
    double* W = nullptr;
    int64_t ldw = 0;
    int vec = 1;   // b = 32 with 16-byte aligned operands: lane-group kernel
    int nt = 256;  // its CTA size (32, 64, 128, 256)
};
int launch_bsr33_df(const Bsr33DfArgs& a, cudaStream_t s);
// r32 = float(W - (A (x) I_R) x32) with A as (hi, lo) floats, double-float
// sums; x32 and r32 dense (ld b). vec: lane-group kernel when b = 32.
int launch_resid_df(int R, int64_t nodes, const int* rowptr, const int* col, const float* vh, const float* vl,
                    const double* W, int64_t ldw, const float* x32, float* r32, int b, cudaStream_t s,
                    int vec = 1, int nt = 256, const float* dinv = nullptr, float inv_theta = 0.f,
                    float* x1 = nullptr);
// With x1 != nullptr also writes the first semi-iteration step on r32,
// x1 = inv_theta D^-1 r32 (dinv per node, ld b).
// w32 = float(W) and x1 = inv_theta D^-1 w32 in one pass (w32, x1 dense).
int launch_convert_x1(int R, int64_t nodes, int b, const double* W, int64_t ldw, float* w32, float inv_theta,
                      const float* dinv, float* x1, cudaStream_t s);

// Y[i, c] = alpha * X[i, c] (rows x b, row-major with leading dims).
template <typename T>
int launch_scale_copy(int64_t rows, int b, T alpha, const T* X, int64_t ldx, T* Y, int64_t ldy,
                      cudaStream_t s);
// Y[i, c] = X[i, c] converted between float and double.
template <typename Tin, typename Tout>
int launch_convert(int64_t rows, int b, const Tin* X, int64_t ldx, Tout* Y, int64_t ldy,
                   cudaStream_t s);
int launch_d2f(int64_t n, const double* x, float* y, cudaStream_t s);
// out[c] += sum_i X[i, c]^2 (out zeroed by the caller).
int launch_colnorm2(int64_t rows, int b, const double* X, int64_t ldx, double* out,
                    cudaStream_t s);
// R[i, c] = KX[i, c] - lam[c] * MX[i, c]
int launch_resid_block(int64_t rows, int b, const double* KX, const double* MX,
                       const double* lam, double* R, cudaStream_t s);
// Philox-4x32-10 Gaussian block (Box-Muller), counter = element index.
int launch_philox_normal(int64_t count, uint64_t seed, double* out, cudaStream_t s);

}  // namespace nm
