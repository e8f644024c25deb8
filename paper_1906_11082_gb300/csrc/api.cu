// C ABI entry points (see include/nm.h for the contract of each call).
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "kernels.h"
#include "nm_internal.h"

namespace nm {

int assemble(nm_ctx* ctx, const nm_mesh* mesh, const nm_model* mdl, nm_problem* P);
int ensure_f32(nm_problem* P, cudaStream_t s);
template <typename T>
int filter_apply_t(nm_problem* P, const nm_filter* f, const T* Y, int64_t ldy, T* Z, int64_t ldz, int b,
                   cudaStream_t s);
template <typename T>
int apply_K_pub(nm_problem* P, const T* X, int64_t ldx, T* Y, int64_t ldy, int b, int k_P, cudaStream_t s);
template <typename T>
int apply_M_pub(nm_problem* P, const T* X, int64_t ldx, T* Y, int64_t ldy, int b, int mode, const double* sk,
                cudaStream_t s);
template <typename T>
int solve_M_pub(nm_problem* P, int k_M, double lo, double hi, const T* W, int64_t ldw, T* X, int64_t ldx,
                int b, cudaStream_t s);
int filter_apply_mixed_pub(nm_problem* P, const nm_filter* f, const double* Y, int64_t ldy, double* Z, int64_t ldz,
                           int b, cudaStream_t s);
int apply_K_mixed_pub(nm_problem* P, const double* X, int64_t ldx, double* Y, int64_t ldy, int b, int k_P,
                      cudaStream_t s);
int solve_M_mixed_pub(nm_problem* P, int k_M, const double* W, int64_t ldw, double* X, int64_t ldx, int b,
                      cudaStream_t s);
void jackson_step_coeffs(double lam_lo, double lam_hi, double xi, double eta, int d, double* gamma, double* c,
                         double* e);
int spectrum_bounds(nm_problem* P, int steps, int k_M, uint64_t seed, double* lam_lo, double* lam_hi);
int lanczos_slice(nm_problem* P, const nm_slice_opts* o, nm_result** out);
int lanczos_multi(nm_problem* P, const nm_slice_opts* o, int S, const double* lam_lo_in, const double* lam_hi_in,
                  nm_result** out);
int lanczos_begin(nm_problem* P, const nm_slice_opts* o, int S, const double* lam_lo_in, const double* lam_hi_in,
                  nm_lanczos** out);
int lanczos_step(nm_lanczos* L, int* active_out);
int lanczos_finish(nm_lanczos* L, nm_result** out);
int lanczos_state(const nm_lanczos* L, int slice, nm_lanczos_info* out);
int lanczos_take(nm_lanczos* L, int q, nm_result** out);
int lanczos_add(nm_lanczos* L, double lam_lo, double lam_hi, uint64_t seed, const double* start, int* index);
void lanczos_free(nm_lanczos* L);
nm_ctx* lanczos_ctx(const nm_lanczos* L);
int ritz(nm_problem* P, nm_ritz_mode mode, const double* V, int64_t ldv, int m, const double* lam_e,
         nm_result** out);
int profile_read(nm_problem* P, int kind, int64_t* launches, double* ms);
int set_tile_rows(nm_problem* P, int64_t rows);
int autotune(nm_problem* P, int b, nm_prec prec, int k_M, std::string* report);
int profile_set(nm_problem* P, int enable, int reset);

uint64_t launches_so_far();

static thread_local nm_ctx* t_ctx = nullptr;
static std::mutex g_err_mu;
static std::string g_last_error;

void set_thread_ctx(nm_ctx* ctx) { t_ctx = ctx; }

int fail(int code, const std::string& msg) {
    if (t_ctx) t_ctx->last_error = msg;
    std::lock_guard<std::mutex> lk(g_err_mu);
    g_last_error = msg;
    return code;
}

int DevBuf::alloc(size_t nbytes) {
    release();
    if (nbytes == 0) nbytes = 1;
    cudaError_t e = cudaMalloc(&p, nbytes);
    if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? NM_ENOMEM : NM_ECUDA,
                    std::string("cudaMalloc(") + std::to_string(nbytes) + "): " + cudaGetErrorString(e));
    }
    bytes = nbytes;
    return NM_OK;
}

void DevBuf::release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
}

}  // namespace nm

using namespace nm;

namespace {

struct CtxScope {
    explicit CtxScope(nm_ctx* c) {
        set_thread_ctx(c);
        if (c) cudaSetDevice(c->device);
    }
    ~CtxScope() { set_thread_ctx(nullptr); }
};

int check_block(const void* X, int64_t ldx, int b, int64_t rows) {
    if (b < 1 || b > 64) return fail(NM_EINVAL, "block width b must be in 1..64");
    if (ldx < b) return fail(NM_EINVAL, "leading dimension must be >= b");
    if (rows > 0 && !X) return fail(NM_EINVAL, "null device pointer");
    return NM_OK;
}

}  // namespace

extern "C" {

int nm_ctx_create(int device, nm_ctx** out) {
    if (!out) return fail(NM_EINVAL, "out is null");
    *out = nullptr;
    nm_ctx* c = new (std::nothrow) nm_ctx();
    if (!c) return fail(NM_ENOMEM, "host allocation failed");
    c->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) {
        delete c;
        return fail(NM_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    }
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cublasCreate(&c->cublas) != CUBLAS_STATUS_SUCCESS ||
        cusolverDnCreate(&c->cusolver) != CUSOLVER_STATUS_SUCCESS) {
        nm_ctx_destroy(c);
        return fail(NM_ECUDA, "failed to create stream / cuBLAS / cuSOLVER handles");
    }
    cublasSetStream(c->cublas, c->stream);
    cusolverDnSetStream(c->cusolver, c->stream);
    *out = c;
    return NM_OK;
}

int nm_ctx_destroy(nm_ctx* c) {
    if (!c) return NM_OK;
    cudaSetDevice(c->device);
    if (c->cusolver) cusolverDnDestroy(c->cusolver);
    if (c->cublas) cublasDestroy(c->cublas);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return NM_OK;
}

const char* nm_last_error(const nm_ctx* c) {
    if (c) return c->last_error.c_str();
    return g_last_error.c_str();
}

int nm_assemble(nm_ctx* ctx, const nm_mesh* mesh, const nm_model* model, nm_problem** out) {
    if (!ctx || !mesh || !model || !out) return fail(NM_EINVAL, "null argument");
    CtxScope sc(ctx);
    *out = nullptr;
    nm_problem* P = new (std::nothrow) nm_problem();
    if (!P) return fail(NM_ENOMEM, "host allocation failed");
    P->ctx = ctx;
    int rc = assemble(ctx, mesh, model, P);
    if (rc != NM_OK) {
        delete P;
        return rc;
    }
    *out = P;
    return NM_OK;
}

int nm_problem_free(nm_problem* P) {
    if (!P) return NM_OK;
    CtxScope sc(P->ctx);
    cudaStreamSynchronize(P->ctx->stream);
    delete P;
    return NM_OK;
}

int nm_problem_get_info(const nm_problem* P, nm_problem_info* info) {
    if (!P || !info) return fail(NM_EINVAL, "null argument");
    *info = P->info;
    return NM_OK;
}

int nm_problem_unodes(const nm_problem* P, int64_t* canon, int64_t* p2, int64_t* pcanon) {
    if (!P) return fail(NM_EINVAL, "null problem");
    if (canon) std::memcpy(canon, P->canon_of_internal.data(), P->canon_of_internal.size() * sizeof(int64_t));
    if (p2) std::memcpy(p2, P->p2_of_internal.data(), P->p2_of_internal.size() * sizeof(int64_t));
    if (pcanon && !P->pcanon_of_internal.empty())
        std::memcpy(pcanon, P->pcanon_of_internal.data(), P->pcanon_of_internal.size() * sizeof(int64_t));
    return NM_OK;
}

int nm_problem_export(const nm_problem* P, int which, int64_t* nrows, int64_t* nnz, int64_t* rowptr,
                      int32_t* col, double* vals) {
    if (!P || !nrows || !nnz) return fail(NM_EINVAL, "null argument");
    CtxScope sc(P->ctx);
    const DevCSR* A = nullptr;
    switch (which) {
        case 0: A = &P->AG; break;
        case 1: A = &P->Mr; break;
        case 2: A = &P->Pn; break;
        case 3: A = &P->EG; break;
        case 4: A = &P->EGt; break;
        default: return fail(NM_EINVAL, "which must be 0..4");
    }
    *nrows = A->nrows;
    *nnz = A->nnz;
    if (!rowptr && !col && !vals) return NM_OK;
    if (rowptr)
        for (int64_t i = 0; i <= A->nrows; ++i) rowptr[i] = A->h_rowptr.empty() ? 0 : A->h_rowptr[i];
    if (col && A->nnz) std::memcpy(col, A->h_col.data(), A->nnz * sizeof(int32_t));
    if (vals && A->nnz) {
        cudaError_t e = cudaMemcpy(vals, A->val.p, A->nnz * A->rb * A->cb * sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return fail(NM_ECUDA, cudaGetErrorString(e));
    }
    return NM_OK;
}

int nm_set_option(nm_problem* P, const char* key, int64_t value) {
    if (!P || !key) return fail(NM_EINVAL, "null argument");
    CtxScope sc(P->ctx);
    P->have_bounds = 0;   // the stored spectrum bounds are recomputed under the new option
    if (std::string(key) == "tile_rows") {
        cudaStreamSynchronize(P->ctx->stream);
        return set_tile_rows(P, value);
    }
    if (std::string(key) == "sched") {
        if (value != 0 && value != 1) return fail(NM_EINVAL, "sched must be 0 or 1");
        P->use_sched = (int)value;
        return NM_OK;
    }
    if (std::string(key) == "dense_tc") {
        if (value != 0 && value != 1) return fail(NM_EINVAL, "dense_tc must be 0 or 1");
        P->ctx->dense_tc = (int)value;
        return NM_OK;
    }
    if (std::string(key) == "tma") {
        if (value != 0 && value != 1) return fail(NM_EINVAL, "tma must be 0 or 1");
        P->use_tma = (int)value;
        return NM_OK;
    }
    if (std::string(key) == "vec") {
        if (value != 0 && value != 1) return fail(NM_EINVAL, "vec must be 0 or 1");
        P->use_vec = (int)value;
        return NM_OK;
    }
    if (std::string(key) == "vec_threads" || std::string(key) == "vec_threads_p") {
        if (value != 32 && value != 64 && value != 128 && value != 256 && value != 512 && value != 1024)
            return fail(NM_EINVAL, std::string(key) + " must be 32, 64, 128, 256, 512 or 1024");
        (std::string(key) == "vec_threads" ? P->vec_threads : P->vec_threads_p) = (int)value;
        return NM_OK;
    }
    if (std::string(key) == "graphs") {
        if (value != 0 && value != 1) return fail(NM_EINVAL, "graphs must be 0 or 1");
        P->use_graphs = (int)value;
        return NM_OK;
    }
    if (std::string(key) == "overlap") {
        if (value != 0 && value != 1) return fail(NM_EINVAL, "overlap must be 0 or 1");
        P->overlap = (int)value;
        return NM_OK;
    }
    if (std::string(key) == "df_threads") {
        if (value != 32 && value != 64 && value != 128 && value != 256)
            return fail(NM_EINVAL, "df_threads must be 32, 64, 128 or 256");
        P->df_threads = (int)value;
        return NM_OK;
    }
    if (std::string(key) == "chunk") {
        if (value != 0 && value != 256 && value != 512 && value != 1024)
            return fail(NM_EINVAL, "chunk must be 0, 256, 512 or 1024");
        P->use_chunk = (int)value;
        return NM_OK;
    }
    if (std::string(key) == "double_float") {
        if (value != 0 && value != 1) return fail(NM_EINVAL, "double_float must be 0 or 1");
        P->use_df = (int)value;
        return NM_OK;
    }
    if (std::string(key) == "tile_kernel") {
        if (value != 1 && value != 2) return fail(NM_EINVAL, "tile_kernel must be 1 or 2");
        P->Mr.tile_kernel = P->Pn.tile_kernel = (int)value;
        return NM_OK;
    }
    return fail(NM_EINVAL, std::string("unknown option: ") + key);
}

int nm_autotune(nm_problem* P, int b, nm_prec prec, int k_M, char* report, int report_len) {
    if (!P) return fail(NM_EINVAL, "null problem");
    CtxScope sc(P->ctx);
    std::string rep;
    NM_TRY(autotune(P, b, prec, k_M, &rep));
    if (report && report_len > 0) {
        const size_t m = std::min<size_t>(rep.size(), (size_t)report_len - 1);
        std::memcpy(report, rep.data(), m);
        report[m] = 0;
    }
    return NM_OK;
}

int nm_problem_gravity(const nm_problem* P, double* g) {
    if (!P || !g) return fail(NM_EINVAL, "null argument");
    CtxScope sc(P->ctx);
    cudaError_t e = cudaMemcpy(g, P->g.p, 3 * P->info.Nu * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(NM_ECUDA, cudaGetErrorString(e));
    return NM_OK;
}

int nm_apply_K(nm_problem* P, const void* X, int64_t ldx, void* Y, int64_t ldy, int b, int k_P, nm_prec prec,
               void* stream) {
    if (!P) return fail(NM_EINVAL, "null problem");
    CtxScope sc(P->ctx);
    NM_TRY(check_block(X, ldx, b, P->info.n));
    NM_TRY(check_block(Y, ldy, b, P->info.n));
    if (k_P <= 0) k_P = 80;
    if (k_P < 2 && P->info.Np) return fail(NM_EINVAL, "k_P must be >= 2");
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == NM_F64) return apply_K_pub<double>(P, (const double*)X, ldx, (double*)Y, ldy, b, k_P, s);
    if (prec == NM_MIXED) return apply_K_mixed_pub(P, (const double*)X, ldx, (double*)Y, ldy, b, k_P, s);
    NM_TRY(ensure_f32(P, s));
    return apply_K_pub<float>(P, (const float*)X, ldx, (float*)Y, ldy, b, k_P, s);
}

int nm_apply_M(nm_problem* P, const void* X, int64_t ldx, void* Y, int64_t ldy, int b, nm_prec prec, void* stream) {
    if (!P) return fail(NM_EINVAL, "null problem");
    CtxScope sc(P->ctx);
    NM_TRY(check_block(X, ldx, b, P->info.n));
    NM_TRY(check_block(Y, ldy, b, P->info.n));
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == NM_F64)
        return apply_M_pub<double>(P, (const double*)X, ldx, (double*)Y, ldy, b, KRON_PLAIN, nullptr, s);
    NM_TRY(ensure_f32(P, s));
    return apply_M_pub<float>(P, (const float*)X, ldx, (float*)Y, ldy, b, KRON_PLAIN, nullptr, s);
}

int nm_apply_R(nm_problem* P, const void* X, int64_t ldx, void* Y, int64_t ldy, int b, nm_prec prec, void* stream) {
    if (!P) return fail(NM_EINVAL, "null problem");
    CtxScope sc(P->ctx);
    NM_TRY(check_block(X, ldx, b, P->info.n));
    NM_TRY(check_block(Y, ldy, b, P->info.n));
    cudaStream_t s = (cudaStream_t)stream;
    const double* O = P->Omega;
    const double sk[9] = {0, -O[2], O[1], O[2], 0, -O[0], -O[1], O[0], 0};
    if (prec == NM_F64) return apply_M_pub<double>(P, (const double*)X, ldx, (double*)Y, ldy, b, KRON_CORI, sk, s);
    NM_TRY(ensure_f32(P, s));
    return apply_M_pub<float>(P, (const float*)X, ldx, (float*)Y, ldy, b, KRON_CORI, sk, s);
}

int nm_solve_M(nm_problem* P, int k_M, double m_lo, double m_hi, const void* W, int64_t ldw, void* X, int64_t ldx,
               int b, nm_prec prec, void* stream) {
    if (!P) return fail(NM_EINVAL, "null problem");
    CtxScope sc(P->ctx);
    NM_TRY(check_block(W, ldw, b, P->info.n));
    NM_TRY(check_block(X, ldx, b, P->info.n));
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == NM_F64)
        return solve_M_pub<double>(P, k_M, m_lo, m_hi, (const double*)W, ldw, (double*)X, ldx, b, s);
    if (prec == NM_MIXED) {
        if (m_lo > 0 || m_hi > 0) return fail(NM_EUNSUPPORTED, "mixed mode uses the P2 element bounds");
        if (k_M < 1) return fail(NM_EINVAL, "k_M must be >= 1");
        return solve_M_mixed_pub(P, k_M, (const double*)W, ldw, (double*)X, ldx, b, s);
    }
    NM_TRY(ensure_f32(P, s));
    return solve_M_pub<float>(P, k_M, m_lo, m_hi, (const float*)W, ldw, (float*)X, ldx, b, s);
}

int nm_set_interval(nm_problem* P, double lo, double hi, nm_unit unit) {
    if (!P) return fail(NM_EINVAL, "null problem");
    if (!(hi > lo) || !std::isfinite(lo) || !std::isfinite(hi)) return fail(NM_EINVAL, "need finite lo < hi");
    if (unit == NM_UNIT_OMEGA) {
        if (hi <= 0) return fail(NM_EINVAL, "omega interval needs hi > 0");
        P->lo = lo > 0 ? lo * lo : 0.0;
        P->hi = hi * hi;
    } else if (unit == NM_UNIT_OMEGA2) {
        P->lo = lo;
        P->hi = hi;
    } else {
        return fail(NM_EINVAL, "unknown unit");
    }
    P->have_interval = 1;
    return NM_OK;
}

int nm_spectrum_bounds(nm_problem* P, int steps, int k_M, uint64_t seed, double* lam_lo, double* lam_hi) {
    if (!P || !lam_lo || !lam_hi) return fail(NM_EINVAL, "null argument");
    CtxScope sc(P->ctx);
    return spectrum_bounds(P, steps, k_M, seed, lam_lo, lam_hi);
}

int nm_filter_design(double lam_lo, double lam_hi, double xi, double eta, int degree, double* gamma, double* c,
                     double* e) {
    if (!gamma || !c || !e || degree < 0) return fail(NM_EINVAL, "bad filter design arguments");
    if (!(lam_hi > lam_lo) || !(eta > xi)) return fail(NM_EINVAL, "need lam_lo < lam_hi and xi < eta");
    jackson_step_coeffs(lam_lo, lam_hi, xi, eta, degree, gamma, c, e);
    return NM_OK;
}

int nm_filter_apply(nm_problem* P, const nm_filter* f, const void* Y, int64_t ldy, void* Z, int64_t ldz, int b,
                    nm_prec prec, void* stream) {
    if (!P || !f) return fail(NM_EINVAL, "null argument");
    CtxScope sc(P->ctx);
    NM_TRY(check_block(Y, ldy, b, P->info.n));
    NM_TRY(check_block(Z, ldz, b, P->info.n));
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == NM_F64)
        return filter_apply_t<double>(P, f, (const double*)Y, ldy, (double*)Z, ldz, b, s);
    if (prec == NM_MIXED) return filter_apply_mixed_pub(P, f, (const double*)Y, ldy, (double*)Z, ldz, b, s);
    NM_TRY(ensure_f32(P, s));
    return filter_apply_t<float>(P, f, (const float*)Y, ldy, (float*)Z, ldz, b, s);
}

int nm_lanczos_slice(nm_problem* P, const nm_slice_opts* opts, nm_result** out) {
    if (!P || !opts || !out) return fail(NM_EINVAL, "null argument");
    CtxScope sc(P->ctx);
    *out = nullptr;
    return lanczos_slice(P, opts, out);
}

// Interval of slice i in lambda (unit conversion as in nm_set_interval).
static int slice_lambda(int nslices, const double* lo, const double* hi, nm_unit unit, std::vector<double>& l,
                        std::vector<double>& u) {
    l.resize(nslices);
    u.resize(nslices);
    for (int i = 0; i < nslices; ++i) {
        if (!(hi[i] > lo[i]) || !std::isfinite(lo[i]) || !std::isfinite(hi[i]))
            return fail(NM_EINVAL, "each slice needs finite lo < hi");
        if (unit == NM_UNIT_OMEGA) {
            if (hi[i] <= 0) return fail(NM_EINVAL, "omega interval needs hi > 0");
            l[i] = lo[i] > 0 ? lo[i] * lo[i] : 0.0;
            u[i] = hi[i] * hi[i];
        } else if (unit == NM_UNIT_OMEGA2) {
            l[i] = lo[i];
            u[i] = hi[i];
        } else {
            return fail(NM_EINVAL, "unknown unit");
        }
    }
    return NM_OK;
}

int nm_lanczos_multi(nm_problem* P, const nm_slice_opts* opts, int nslices, const double* lo, const double* hi,
                     nm_unit unit, nm_result** out) {
    if (!P || !opts || !out || !lo || !hi || nslices < 1) return fail(NM_EINVAL, "bad argument");
    CtxScope sc(P->ctx);
    for (int i = 0; i < nslices; ++i) out[i] = nullptr;
    std::vector<double> l, u;
    NM_TRY(slice_lambda(nslices, lo, hi, unit, l, u));
    return lanczos_multi(P, opts, nslices, l.data(), u.data(), out);
}

int nm_lanczos_begin(nm_problem* P, const nm_slice_opts* opts, int nslices, const double* lo, const double* hi,
                     nm_unit unit, nm_lanczos** out) {
    if (!P || !opts || !out) return fail(NM_EINVAL, "null argument");
    CtxScope sc(P->ctx);
    *out = nullptr;
    std::vector<double> l, u;
    if (nslices == 0) {
        if (!P->have_interval) return fail(NM_EINVAL, "call nm_set_interval first (or pass the slices)");
        l.assign(1, P->lo);
        u.assign(1, P->hi);
        nslices = 1;
    } else {
        if (nslices < 0 || !lo || !hi) return fail(NM_EINVAL, "bad slice list");
        NM_TRY(slice_lambda(nslices, lo, hi, unit, l, u));
    }
    return lanczos_begin(P, opts, nslices, l.data(), u.data(), out);
}

int nm_lanczos_step(nm_lanczos* L, int* active) {
    if (!L || !active) return fail(NM_EINVAL, "null argument");
    CtxScope sc(lanczos_ctx(L));
    return lanczos_step(L, active);
}

int nm_lanczos_get_info(const nm_lanczos* L, int slice, nm_lanczos_info* info) {
    if (!L || !info) return fail(NM_EINVAL, "null argument");
    return lanczos_state(L, slice, info);
}

int nm_lanczos_finish(nm_lanczos* L, nm_result** out) {
    if (!L || !out) return fail(NM_EINVAL, "null argument");
    CtxScope sc(lanczos_ctx(L));
    return lanczos_finish(L, out);
}

int nm_lanczos_add(nm_lanczos* L, double lo, double hi, nm_unit unit, uint64_t seed, const double* start,
                   int* index) {
    if (!L || !index) return fail(NM_EINVAL, "null argument");
    CtxScope sc(lanczos_ctx(L));
    std::vector<double> l, u;
    NM_TRY(slice_lambda(1, &lo, &hi, unit, l, u));
    return lanczos_add(L, l[0], u[0], seed, start, index);
}

int nm_lanczos_take(nm_lanczos* L, int slice, nm_result** out) {
    if (!L || !out) return fail(NM_EINVAL, "null argument");
    CtxScope sc(lanczos_ctx(L));
    return lanczos_take(L, slice, out);
}

int nm_lanczos_free(nm_lanczos* L) {
    if (!L) return NM_OK;
    lanczos_free(L);   // touches only the run's own buffers, not its problem
    return NM_OK;
}

int nm_ritz(nm_problem* P, nm_ritz_mode mode, const double* V, int64_t ldv, int m, const double* lam_e,
            nm_result** out) {
    if (!P || !out) return fail(NM_EINVAL, "null argument");
    CtxScope sc(P->ctx);
    *out = nullptr;
    return ritz(P, mode, V, ldv, m, lam_e, out);
}

int nm_gemm_tn(nm_ctx* ctx, int64_t I, int64_t J, int64_t K, double alpha, const double* X, int64_t ldx,
               const double* Y, int64_t ldy, double beta, double* C, int64_t ldc, void* stream) {
    if (!ctx) return fail(NM_EINVAL, "null context");
    CtxScope sc(ctx);
    if (I < 0 || J < 0 || K < 0) return fail(NM_EINVAL, "negative size");
    if (I == 0 || J == 0) return NM_OK;
    if (!C || ldc < I || (K > 0 && (!X || !Y || ldx < I || ldy < J)))
        return fail(NM_EINVAL, "null operand or leading dimension too small");
    return ozaki_gemm_tn(ctx, (cudaStream_t)stream, I, J, K, alpha, X, ldx, Y, ldy, beta, C, ldc);
}

int nm_gemm_nn(nm_ctx* ctx, int64_t I, int64_t J, int64_t K, double alpha, const double* X, int64_t ldx,
               const double* Y, int64_t ldy, double beta, double* D, int64_t ldd, void* stream) {
    if (!ctx) return fail(NM_EINVAL, "null context");
    CtxScope sc(ctx);
    if (I < 0 || J < 0 || K < 0) return fail(NM_EINVAL, "negative size");
    if (I == 0 || J == 0) return NM_OK;
    if (!D || ldd < J || (K > 0 && (!X || !Y || ldx < K || ldy < K)))
        return fail(NM_EINVAL, "null operand or leading dimension too small");
    return ozaki_gemm_nn((cudaStream_t)stream, I, J, K, alpha, X, ldx, Y, ldy, beta, D, ldd);
}

int nm_profile(nm_problem* P, int enable, int reset) {
    if (!P) return fail(NM_EINVAL, "null problem");
    CtxScope sc(P->ctx);
    return profile_set(P, enable, reset);
}

uint64_t nm_kernel_launches(void) { return launches_so_far(); }

int nm_profile_read(nm_problem* P, int kind, int64_t* launches, double* ms) {
    if (!P || !launches || !ms) return fail(NM_EINVAL, "null argument");
    if (kind < 0 || kind > 2) return fail(NM_EINVAL, "kind must be 0, 1 or 2");
    CtxScope sc(P->ctx);
    return profile_read(P, kind, launches, ms);
}

int nm_result_get_info(const nm_result* R, nm_result_info* info) {
    if (!R || !info) return fail(NM_EINVAL, "null argument");
    *info = R->info;
    return NM_OK;
}

int nm_result_values(const nm_result* R, double* lambda, double* resid) {
    if (!R) return fail(NM_EINVAL, "null result");
    if (lambda && !R->lambda.empty()) std::memcpy(lambda, R->lambda.data(), R->lambda.size() * sizeof(double));
    if (resid && !R->resid.empty()) std::memcpy(resid, R->resid.data(), R->resid.size() * sizeof(double));
    return NM_OK;
}

const void* nm_result_vectors(const nm_result* R) { return R ? R->X.p : nullptr; }

int nm_result_free(nm_result* R) {
    delete R;
    return NM_OK;
}

}  // extern "C"
