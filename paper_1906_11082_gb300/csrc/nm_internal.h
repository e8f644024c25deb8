// Internal structures of the nm library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cublas_v2.h>
#include <cusolverDn.h>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/nm.h"
#include "kernels.h"

namespace nm {

// Error propagation inside the library: every failing call sets the
// context message and returns a code; nothing throws across the ABI.
struct Status {
    int code = NM_OK;
    std::string msg;
};

#define NM_CUDA(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return ::nm::fail(NM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define NM_CUBLAS(call)                                                                    \
    do {                                                                                   \
        cublasStatus_t s_ = (call);                                                        \
        if (s_ != CUBLAS_STATUS_SUCCESS)                                                   \
            return ::nm::fail(NM_ECUDA, std::string(#call) + ": cublas status " +           \
                                            std::to_string((int)s_));                      \
    } while (0)

#define NM_CUSOLVER(call)                                                                  \
    do {                                                                                   \
        cusolverStatus_t s_ = (call);                                                      \
        if (s_ != CUSOLVER_STATUS_SUCCESS)                                                 \
            return ::nm::fail(NM_ECUDA, std::string(#call) + ": cusolver status " +         \
                                            std::to_string((int)s_));                      \
    } while (0)

#define NM_TRY(expr)                 \
    do {                             \
        int r_ = (expr);             \
        if (r_ != NM_OK) return r_;  \
    } while (0)

int fail(int code, const std::string& msg);   // records msg for nm_last_error
void set_thread_ctx(nm_ctx* ctx);

// Device buffer owned by the library.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    int alloc(size_t nbytes);
    void release();
    template <class T> T* as() const { return static_cast<T*>(p); }
    ~DevBuf() { release(); }
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
};

// Sparse matrices on the device. Block CSR with rb x cb blocks, values
// row-major inside a block, stored in double and (lazily) in float.
struct DevCSR {
    int64_t nrows = 0, ncols = 0, nnz = 0;
    int rb = 1, cb = 1;
    DevBuf rowptr;   // int32 [nrows + 1]  (nnz < 2^31 checked at build)
    DevBuf col;      // int32 [nnz]
    DevBuf val;      // double [nnz * rb * cb]
    DevBuf val32;    // float  [nnz * rb * cb] (on demand): fl(val), the high part
    DevBuf vlo32;    // float  [nnz * rb * cb] (on demand): fl(val - fl(val)), the low part
    DevBuf dinv;     // inverse diagonal (scalar square matrices only), double
    DevBuf dinv32;
    std::vector<int32_t> h_rowptr, h_col;   // host copy of the pattern
    // Row tiles for shared-memory staging of the gathered operand: tile t
    // holds rows [t*tile_rows, (t+1)*tile_rows); its distinct columns are
    // tile_ucol[tile_uptr[t] .. tile_uptr[t+1]) and lcol[e] is the position
    // of col[e] in its tile's list (scalar square matrices only).
    int tile_rows = 0;
    int64_t ntiles = 0;
    int tile_umax = 0;
    int tile_kernel = 2;
    DevBuf tile_uptr;  // int32 [ntiles + 1]
    DevBuf tile_ucol;  // int32
    DevBuf lcol;       // uint16 [nnz]
    // row tiles of the bulk-copy staged float mass step (mass_tma.cu),
    // built on first use: state 0 not built, 1 built, -1 not eligible
    int tma_state = 0;
    TmaTiles tma;
    DevBuf tma_desc, tma_ucol, tma_lcol, tma_vals, tma_rowptr, tma_dinv, tma_ldiag, tma_err;
};

int build_tma_tiles(DevCSR& A, cudaStream_t s);

struct Workspace {
    DevBuf buf;      // filter recurrence scratch
    size_t bytes = 0;
};

// Self-gravitation (selfgrav.cu): charges C (points x dofs, CSR), its
// transpose, the charge points and their inverse self distances, and the
// point-sized scratch of one block of up to 64 columns.
struct SelfGravity {
    int on = 0;
    int64_t np = 0;
    double G = 0;
    DevBuf pts, invR;                 // double [3 np], [np]
    DevBuf c_rp, c_col, c_val;        // C: int64 [np + 1], int32, double
    DevBuf t_rp, t_col, t_val;        // C^T: int64 [n + 1], int32, double
    DevBuf q, phi;                    // double [np * 64]
    DevBuf part;                      // partial sums of split n-body launches (small np)
};

}  // namespace nm

struct nm_ctx {
    int device = 0;
    std::string last_error;
    cublasHandle_t cublas = nullptr;
    cusolverDnHandle_t cusolver = nullptr;
    cudaStream_t stream = nullptr;   // library-owned stream for blocking calls
    nm::DevBuf gemm_ws;              // split parts of the tensor-core dense products
    int dense_tc = 1;                // dense products on the tensor cores (0: cuBLAS DGEMM)
};

namespace nm {
// FP64-accurate dense products on the tensor cores (ozaki_gemm.cu).
// TN: C (I x J, col-major, ldc) = alpha X^T Y + beta C, X: K x I, Y: K x J row-major.
int ozaki_gemm_tn(nm_ctx* ctx, cudaStream_t s, int64_t I, int64_t J, int64_t K, double alpha, const double* X,
                  int64_t ldx, const double* Y, int64_t ldy, double beta, double* C, int64_t ldc);
// NN: D (I x J, row-major, ldd) = alpha X Y + beta D, X: I x K row-major, Y: K x J col-major.
int ozaki_gemm_nn(cudaStream_t s, int64_t I, int64_t J, int64_t K, double alpha, const double* X, int64_t ldx,
                  const double* Y, int64_t ldy, double beta, double* D, int64_t ldd);
// Self-gravitation (selfgrav.cu). usol / uflu: internal u-node of the
// solid / fluid copy of each P2 node, -1 where the copy does not exist.
int build_self_gravity(nm_problem* P, const double* xyz, const int32_t* tet, const int64_t* tet10,
                       const uint8_t* region, const double* rho, int64_t nt, const int32_t* usol,
                       const int32_t* uflu, double G);
// Its host part: points (x, y, z per point), inverse self distances and the
// entries (point, dof, value) of C, duplicates not summed.
void self_gravity_host(const double* xyz, const int32_t* tet, const int64_t* tet10, const uint8_t* region,
                       const double* rho, int64_t nt, const int32_t* usol, const int32_t* uflu,
                       std::vector<double>& pts, std::vector<double>& invR, std::vector<int64_t>& erow,
                       std::vector<int32_t>& ecol, std::vector<double>& eval);
// W -= C^T S C X, X and W row-major n x b (b <= 64) in double.
int apply_selfgrav(nm_problem* P, const double* X, int64_t ldx, double* W, int64_t ldw, int b, cudaStream_t s);
}  // namespace nm

struct nm_problem {
    nm_ctx* ctx = nullptr;
    nm_problem_info info{};
    // maps (host)
    std::vector<int64_t> canon_of_internal;   // [Nu]
    std::vector<int64_t> p2_of_internal;      // [Nu]
    std::vector<int64_t> pcanon_of_internal;  // [Np]
    // device matrices
    nm::DevCSR AG;     // 3x3 blocks, u x u
    nm::DevCSR Mr;     // scalar, u x u (same pattern as AG)
    nm::DevCSR Pn;     // scalar -A_p, p x p
    nm::DevCSR EG;     // 3x1 blocks, u x p
    nm::DevCSR EGt;    // 1x3 blocks, p x u
    nm::DevBuf g;      // double [Nu * 3] reference field at u-nodes
    nm::SelfGravity sg;  // -C^T S C of the full operator (NM_SELF_GRAVITY)
    double Omega[3] = {0, 0, 0};
    uint32_t flags = 0;
    // slice
    double lo = 0, hi = 0;
    int have_interval = 0;
    double bounds_lo = 0, bounds_hi = 0;
    int have_bounds = 0;
    // (steps, k_M, seed) of the stored bounds; any option change clears have_bounds
    int bounds_key_steps = 0, bounds_key_kM = 0;
    uint64_t bounds_key_seed = 0;
    // kernel timing (nm_profile): event pairs per region kind
    int profile = 0;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_regions;  // kind, (start, stop)
    std::vector<int64_t> ev_launches;   // launches inside each region
    size_t ev_next = 0;
    // mixed form: K_eff SpMM and refinement residuals in double-float
    int use_df = 1;
    // SM-local persistent schedule of the semi-iteration kernels
    int use_sched = 0;
    int use_vec = 1;      // vectorised gathers for float b = 32 blocks
    int use_tma = 0;      // shared-memory staged tiles for the float b = 32 mass steps (option "tma")
    int vec_threads = 32;   // their CTA size (3-component rows)
    int vec_threads_p = 128;  // ... and for the 1-component pressure rows
    int df_threads = 32;    // CTA size of the lane-group double-float kernels
    int use_chunk = 0;    // threads per CTA of the chunked row schedule, 0 = off
    nm::DevBuf sched;   // int [nreg] region counters
    int nreg = 0;
    // scratch for the filter recurrence
    nm::Workspace ws;
    nm::DevBuf pscratch;     // pressure-sized scratch for the Schur term
    // mixed-form K_eff: the fluid pressure chain runs on `aux` (high
    // priority) while A_G X runs on the caller's stream (option "overlap")
    int overlap = 0;
    // mixed-form filter degrees 1..d-1 replayed as two captured CUDA graphs
    // (option "graphs"): gamma table and degree counter live on the device
    int use_graphs = 0;
    nm::DevBuf graph_gam;   // (degree + 1) doubles
    nm::DevBuf graph_deg;   // one int
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    ~nm_problem() {
        for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (aux) cudaStreamDestroy(aux);
    }
};

namespace nm {
// Begin / end a timed launch region on stream s (no-ops unless profiling).
int prof_begin(nm_problem* P, cudaStream_t s, cudaEvent_t* start);
int prof_end(nm_problem* P, cudaStream_t s, int kind, cudaEvent_t start, int64_t launches);
}  // namespace nm

struct nm_result {
    nm_result_info info{};
    std::vector<double> lambda, resid;
    nm::DevBuf X;
};
