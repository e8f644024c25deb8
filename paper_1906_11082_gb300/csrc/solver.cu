// Filter recurrence, operator pieces, spectrum bounds, filtered block
// Lanczos, Rayleigh-Ritz and the rotating projection (paper Sec. 6.2, 7).
//
// All vectors stay on the device; the host only sequences launches and
// reads small results (Ritz values, residual norms) at convergence tests.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <memory>
#include <cstdio>
#include <cstring>
#include <deque>
#include <vector>

#include "kernels.h"
#include "nm_internal.h"

namespace nm {

int ensure_f32(nm_problem* P, cudaStream_t s);
int ensure_df(nm_problem* P, cudaStream_t s);
template <typename T>
int filter_apply_t(nm_problem* P, const nm_filter* f, const T* Y, int64_t ldy, T* Z, int64_t ldz, int b, cudaStream_t s);
struct GammaTable;
static int filter_apply_mixed(nm_problem* P, const nm_filter* f, const double* Y, int64_t ldy, double* Z,
                              int64_t ldz, int b, cudaStream_t s, const GammaTable* gt = nullptr);

static const double kMassLo = 0.25;
static const double kMassHi = (19.0 + 15.779733838059499) / 8.0;   // (19 + sqrt(249)) / 8

template <typename T>
struct Mats {
    int64_t Nu = 0, Np = 0;
    const int *u_rp = nullptr, *u_col = nullptr;
    const T *AG = nullptr, *Mr = nullptr, *dM = nullptr;
    const int *p_rp = nullptr, *p_col = nullptr;
    const T *Pn = nullptr, *dP = nullptr;
    const int *e_rp = nullptr, *e_col = nullptr;
    const T* EG = nullptr;
    const int *et_rp = nullptr, *et_col = nullptr;
    const T* EGt = nullptr;
    const DevCSR* Mcsr = nullptr;
    const DevCSR* Pcsr = nullptr;
    nm_problem* P = nullptr;
};

template <typename T>
static const T* vals(const DevCSR& A);
template <>
const double* vals<double>(const DevCSR& A) { return A.val.as<double>(); }
template <>
const float* vals<float>(const DevCSR& A) { return A.val32.as<float>(); }
template <typename T>
static const T* dinv(const DevCSR& A);
template <>
const double* dinv<double>(const DevCSR& A) { return A.dinv.as<double>(); }
template <>
const float* dinv<float>(const DevCSR& A) { return A.dinv32.as<float>(); }

template <typename T>
static Mats<T> mats(nm_problem* P) {
    Mats<T> m;
    m.Nu = P->info.Nu;
    m.Np = P->info.Np;
    m.u_rp = P->AG.rowptr.as<int>();
    m.u_col = P->AG.col.as<int>();
    m.AG = vals<T>(P->AG);
    m.Mr = vals<T>(P->Mr);
    m.dM = dinv<T>(P->Mr);
    m.Mcsr = &P->Mr;
    m.Pcsr = &P->Pn;
    m.P = P;
    if (m.Np > 0) {
        m.p_rp = P->Pn.rowptr.as<int>();
        m.p_col = P->Pn.col.as<int>();
        m.Pn = vals<T>(P->Pn);
        m.dP = dinv<T>(P->Pn);
        m.e_rp = P->EG.rowptr.as<int>();
        m.e_col = P->EG.col.as<int>();
        m.EG = vals<T>(P->EG);
        m.et_rp = P->EGt.rowptr.as<int>();
        m.et_col = P->EGt.col.as<int>();
        m.EGt = vals<T>(P->EGt);
    }
    return m;
}

template <typename T>
static void set_sched(KronArgs<T>& a, nm_problem* P) {
    a.chunk = P->use_chunk;
    a.vec = P->use_vec;
    a.vec_threads = P->vec_threads;
    a.vec_threads_p = P->vec_threads_p;
    if (P->use_sched && P->sched.p) {
        a.sched = P->sched.as<int>();
        a.nreg = P->nreg;
    }
}

template <typename T>
static void set_tiles(KronArgs<T>& a, const DevCSR& A) {
    a.tile_uptr = A.tile_uptr.as<int>();
    a.tile_ucol = A.tile_ucol.as<int>();
    a.lcol = A.lcol.as<uint16_t>();
    a.tile_rows = A.tile_rows;
    a.ntiles = A.ntiles;
    a.tile_umax = A.tile_umax;
    a.tile_kernel = A.tile_kernel;
}

struct ChebCoef {
    double inv_theta, four_sig2;
    ChebCoef(double lo, double hi) {
        const double th = 0.5 * (hi + lo), de = 0.5 * (hi - lo);
        inv_theta = 1.0 / th;
        four_sig2 = 4.0 * (th / de) * (th / de);
    }
};

// Scratch for one operator application on b columns.
template <typename T>
struct Scratch {
    T *TA, *TB, *W, *XA, *XB;    // n x b each (ld b)
    T *Q, *PA, *PB;              // Np x b each
};

template <typename T>
static int get_scratch(nm_problem* P, int b, Scratch<T>& S) {
    const int64_t n = P->info.n, Np = P->info.Np;
    const size_t need = (size_t)(5 * n + 3 * Np) * b * sizeof(T);
    if (P->ws.bytes < need) {
        P->ws.buf.release();
        NM_TRY(P->ws.buf.alloc(need));
        P->ws.bytes = need;
    }
    T* p = P->ws.buf.as<T>();
    S.TA = p; p += n * b;
    S.TB = p; p += n * b;
    S.W = p; p += n * b;
    S.XA = p; p += n * b;
    S.XB = p; p += n * b;
    S.Q = p; p += Np * b;
    S.PA = p; p += Np * b;
    S.PB = p;
    return NM_OK;
}

// Pressure Schur solve: returns the buffer holding S ~ (-A_p)^{-1} E_G^T X.
template <typename T>
static int schur_pressure(const Mats<T>& m, const T* X, int64_t ldx, int b, int k_P, double lo,
                          double hi, const Scratch<T>& S, const T** out, cudaStream_t s) {
    ChebCoef cc(lo, hi);
    Bsr13Args<T> q;
    q.nrows = (int)m.Np;
    q.rowptr = m.et_rp;
    q.col = m.et_col;
    q.val = m.EGt;
    q.b = b;
    q.X = X;
    q.ldx = ldx;
    q.Q = S.Q;
    q.ldq = b;
    q.S1 = S.PA;
    q.lds1 = b;
    q.dinv = m.dP;
    q.inv_theta = (T)cc.inv_theta;
    NM_TRY(launch_bsr13<T>(q, s));
    T* buf[2] = {S.PB, S.PA};   // buf[1] holds x_1
    double om = 2.0;
    for (int j = 2; j <= k_P; ++j) {
        om = 1.0 / (1.0 - om / cc.four_sig2);
        KronArgs<T> a;
        a.nrows = (int)m.Np;
        a.rowptr = m.p_rp;
        a.col = m.p_col;
        a.val = m.Pn;
        a.dinv = m.dP;
        set_tiles(a, *m.Pcsr);
        set_sched(a, m.P);
        a.b = b;
        a.X = buf[(j - 1) & 1];
        a.ldx = b;
        a.W = S.Q;
        a.ldw = b;
        a.Xp = j == 2 ? nullptr : buf[j & 1];
        a.ldp = b;
        a.Xn = buf[j & 1];
        a.ldn = b;
        a.om = (T)om;
        a.inv_theta = (T)cc.inv_theta;
        NM_TRY(launch_kron<T>(1, KRON_CHEB, a, s));
    }
    *out = buf[k_P & 1];
    return NM_OK;
}

// W = K_eff X (optionally X1 = inv_theta D^-1 W for the mass solve).
template <typename T>
static int apply_K_t(nm_problem* P, const T* X, int64_t ldx, T* W, int64_t ldw, int b, int k_P,
                     const Scratch<T>& S, T* X1, double inv_theta_M, cudaStream_t s) {
    Mats<T> m = mats<T>(P);
    Bsr33Args<T> a;
    a.nrows = (int)m.Nu;
    a.rowptr = m.u_rp;
    a.col = m.u_col;
    a.val = m.AG;
    a.b = b;
    a.X = X;
    a.ldx = ldx;
    a.W = W;
    a.ldw = ldw;
    // with self-gravitation the fused first mass step follows the
    // -C^T S C X correction instead of riding on the A_G product
    const bool sg = P->sg.on != 0;
    if (sg && sizeof(T) != sizeof(double))
        return fail(NM_EUNSUPPORTED, "self-gravitation needs the double or mixed precision path");
    a.X1 = sg ? nullptr : X1;
    a.ldx1 = b;
    a.dinv = m.dM;
    a.inv_theta = (T)inv_theta_M;
    if (m.Np > 0) {
        const T* Sp = nullptr;
        NM_TRY(schur_pressure<T>(m, X, ldx, b, k_P, kMassLo, kMassHi, S, &Sp, s));
        a.e_rowptr = m.e_rp;
        a.e_col = m.e_col;
        a.e_val = m.EG;
        a.S = Sp;
        a.lds = b;
    }
    NM_TRY(launch_bsr33<T>(a, s));
    if (sg) {
        NM_TRY(apply_selfgrav(P, (const double*)X, ldx, (double*)W, ldw, b, s));
        if (X1) NM_TRY(launch_dscale<T>(3, m.Nu, b, (T)inv_theta_M, m.dM, W, ldw, X1, b, s));
    }
    return NM_OK;
}

// Mass-solve semi-iteration steps 2..k_M starting from x_1 in S.XA and the
// right-hand side S.W. With filt != nullptr the last step is fused with
// the outer Chebyshev update; otherwise x_{k_M} is copied to Xout.
// Per-slice gammas of a batched filter: dev[k * S + g] is gamma_k of the
// slice owning column group g (group columns wide); host mirrors it.
struct GammaTable {
    const double* dev;
    const double* host;
    int S;
    int group;
};

struct FiltStep {
    double a1, cshift, a2, gam;
    const double* gam_tab = nullptr;   // device, one gamma per column group
    int gam_group = 1;
};

template <typename T>
static int mass_steps(const Mats<T>& m, int b, int k_M, double lo, double hi, const Scratch<T>& S,
                      const FiltStep* filt, const T* Tk, const T* Tp, T* Tn, T* Z, int64_t ldz,
                      T* Xout, int64_t ldo, cudaStream_t s) {
    ChebCoef cc(lo, hi);
    T* buf[2] = {S.XB, S.XA};
    double om = 2.0;
    for (int j = 2; j <= k_M; ++j) {
        om = 1.0 / (1.0 - om / cc.four_sig2);
        KronArgs<T> a;
        a.nrows = (int)m.Nu;
        a.rowptr = m.u_rp;
        a.col = m.u_col;
        a.val = m.Mr;
        a.dinv = m.dM;
        set_tiles(a, *m.Mcsr);
        set_sched(a, m.P);
        a.b = b;
        a.X = buf[(j - 1) & 1];
        a.ldx = b;
        a.W = S.W;
        a.ldw = b;
        a.Xp = j == 2 ? nullptr : buf[j & 1];
        a.ldp = b;
        a.om = (T)om;
        a.inv_theta = (T)cc.inv_theta;
        if (j == k_M && filt) {
            a.Tk = Tk;
            a.ldtk = b;
            a.Tp = Tp;
            a.ldtp = b;
            a.Tn = Tn;
            a.ldtn = b;
            a.Z = Z;
            a.ldz = ldz;
            a.a1 = (T)filt->a1;
            a.cshift = (T)filt->cshift;
            a.a2 = (T)filt->a2;
            a.gam = (T)filt->gam;
            a.gam_tab = filt->gam_tab;
            a.gam_group = filt->gam_group;
            NM_TRY(launch_kron<T>(3, KRON_CHEB_FILT, a, s));
        } else if (j == k_M && Xout) {
            a.Xn = Xout;
            a.ldn = ldo;
            NM_TRY(launch_kron<T>(3, KRON_CHEB, a, s));
        } else {
            a.Xn = buf[j & 1];
            a.ldn = b;
            NM_TRY(launch_kron<T>(3, KRON_CHEB, a, s));
        }
    }
    return NM_OK;
}

template <typename T>
static int filter_core(nm_problem* P, const nm_filter* f, const T* Y, int64_t ldy, T* Z, int64_t ldz, int b,
                       const GammaTable* gt, cudaStream_t s) {
    const int d = f->degree;
    if (d < 0 || (!f->gamma && !gt)) return fail(NM_EINVAL, "filter needs degree >= 0 and gamma");
    if (f->k_M < 2 || (P->info.Np > 0 && f->k_P < 2)) return fail(NM_EINVAL, "k_M and k_P must be >= 2");
    if (!(f->e > 0)) return fail(NM_EINVAL, "filter half-width e must be positive");
    const double mlo = f->m_lo > 0 ? f->m_lo : kMassLo;
    const double mhi = f->m_hi > 0 ? f->m_hi : kMassHi;
    if (!(mhi > mlo)) return fail(NM_EINVAL, "mass bounds need m_hi > m_lo > 0");
    const int64_t n = P->info.n;
    Scratch<T> S;
    NM_TRY(get_scratch<T>(P, b, S));
    Mats<T> m = mats<T>(P);
    const ChebCoef cc(mlo, mhi);
    if (gt) {
        for (int g = 0; g < gt->S; ++g)
            NM_TRY(launch_scale_copy<T>(n, gt->group, (T)gt->host[g], Y + g * gt->group, ldy, Z + g * gt->group,
                                        ldz, s));
    } else {
        NM_TRY(launch_scale_copy<T>(n, b, (T)f->gamma[0], Y, ldy, Z, ldz, s));
    }
    if (d == 0) return NM_OK;
    NM_TRY(launch_scale_copy<T>(n, b, (T)1, Y, ldy, S.TA, b, s));
    T* cur = S.TA;   // T_k
    T* prev = S.TB;  // T_{k-1}
    const int64_t kl = 1 + (P->info.Np > 0 ? f->k_P : 0);
    for (int k = 0; k < d; ++k) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        NM_TRY(prof_begin(P, s, &e0));
        NM_TRY(apply_K_t<T>(P, cur, b, S.W, b, b, f->k_P, S, S.XA, cc.inv_theta, s));
        NM_TRY(prof_end(P, s, 1, e0, kl));
        NM_TRY(prof_begin(P, s, &e1));
        FiltStep fs;
        fs.cshift = f->c;
        fs.gam = gt ? 0.0 : f->gamma[k + 1];
        if (gt) {
            fs.gam_tab = gt->dev + (int64_t)(k + 1) * gt->S;
            fs.gam_group = gt->group;
        }
        if (k == 0) {
            fs.a1 = 1.0 / f->e;
            fs.a2 = 0.0;
            NM_TRY(mass_steps<T>(m, b, f->k_M, mlo, mhi, S, &fs, cur, nullptr, prev, Z, ldz, nullptr, 0, s));
        } else {
            fs.a1 = 2.0 / f->e;
            fs.a2 = 1.0;
            NM_TRY(mass_steps<T>(m, b, f->k_M, mlo, mhi, S, &fs, cur, prev, prev, Z, ldz, nullptr, 0, s));
        }
        NM_TRY(prof_end(P, s, 0, e1, f->k_M - 1));
        std::swap(cur, prev);
    }
    return NM_OK;
}

// ------------------------------------------------------------------ mixed precision
// Scratch: doubles TA, TB, W (n x b), S64, Q64 (Np x b); floats w32, xa, xb,
// xs, es (n x b; the pressure solve reuses their first Np x b entries).
struct MixScratch {
    double *TA, *TB, *W, *S64, *Q64;
    float *w32, *xa, *xb, *xs, *es;
    float *Th, *Tl;   // double-float split of the block K_eff is applied to
};

static int get_mix_scratch(nm_problem* P, int b, MixScratch& S) {
    const int64_t n = P->info.n, Np = P->info.Np;
    const size_t need = (size_t)(3 * n + 2 * Np) * b * sizeof(double) + (size_t)7 * n * b * sizeof(float);
    if (P->ws.bytes < need) {
        P->ws.buf.release();
        NM_TRY(P->ws.buf.alloc(need));
        P->ws.bytes = need;
    }
    double* d = P->ws.buf.as<double>();
    S.TA = d; d += n * b;
    S.TB = d; d += n * b;
    S.W = d; d += n * b;
    S.S64 = d; d += Np * b;
    S.Q64 = d; d += Np * b;
    float* f = reinterpret_cast<float*>(d);
    S.w32 = f; f += n * b;
    S.xa = f; f += n * b;
    S.xb = f; f += n * b;
    S.xs = f; f += n * b;
    S.es = f; f += n * b;
    S.Th = f; f += n * b;
    S.Tl = f;
    return NM_OK;
}

// k steps of float Jacobi-Chebyshev semi-iteration for (A (x) I_R) x = w;
// w, xa, xb, xout: (R nodes) x b floats with ld b, xout distinct from xa, xb.
static int cheb32(nm_problem* P, const DevCSR& A, int R, int b, int k, double lo, double hi, const float* w,
                  float* xa, float* xb, float* xout, cudaStream_t s, bool x1_ready = false) {
    const ChebCoef cc(lo, hi);
    const int64_t nodes = A.nrows;
    if (k == 1) return launch_dscale<float>(R, nodes, b, (float)cc.inv_theta, A.dinv32.as<float>(), w, b, xout, b, s);
    // x1_ready: the producer of w already wrote the first step into xa
    if (!x1_ready)
        NM_TRY(launch_dscale<float>(R, nodes, b, (float)cc.inv_theta, A.dinv32.as<float>(), w, b, xa, b, s));
    float* buf[2] = {xb, xa};
    double om = 2.0;
    // profile kind 2: the float mass-matrix semi-iteration launches alone
    cudaEvent_t ev = nullptr;
    if (R == 3) NM_TRY(prof_begin(P, s, &ev));
    for (int j = 2; j <= k; ++j) {
        om = 1.0 / (1.0 - om / cc.four_sig2);
        KronArgs<float> a;
        a.nrows = (int)nodes;
        a.rowptr = A.rowptr.as<int>();
        a.col = A.col.as<int>();
        a.val = A.val32.as<float>();
        a.dinv = A.dinv32.as<float>();
        set_tiles(a, A);
        set_sched(a, P);
        a.b = b;
        a.X = buf[(j - 1) & 1];
        a.ldx = b;
        a.W = w;
        a.ldw = b;
        a.Xp = j == 2 ? nullptr : buf[j & 1];
        a.ldp = b;
        a.Xn = j == k ? xout : buf[j & 1];
        a.ldn = b;
        a.om = (float)om;
        a.inv_theta = (float)cc.inv_theta;
        if (R == 3 && b == 32 && P->use_tma && A.tma_state == 1) a.tma = A.tma;
        NM_TRY(launch_kron<float>(R, KRON_CHEB, a, s));
    }
    if (R == 3) NM_TRY(prof_end(P, s, 2, ev, k - 1));
    return NM_OK;
}

// Refined solve: x = P32 w, r = w - A x (double), e = P32 r; leaves x in
// S.xs and e in S.es (the caller combines them).
static int mixed_solve(nm_problem* P, const DevCSR& A, int R, int b, int k, const double* W, int64_t ldw,
                       const MixScratch& S, bool df, cudaStream_t s) {
    const int64_t rows = R * A.nrows;
    const ChebCoef cc(kMassLo, kMassHi);
    const float it = (float)cc.inv_theta;
    // k >= 2: the float conversion of W and the double-float residual also
    // write the first semi-iteration step, so cheb32 starts at step 2
    const bool fuse = k >= 2;
    if (fuse)
        NM_TRY(launch_convert_x1(R, A.nrows, b, W, ldw, S.w32, it, A.dinv32.as<float>(), S.xa, s));
    else
        NM_TRY((launch_convert<double, float>(rows, b, W, ldw, S.w32, b, s)));
    NM_TRY(cheb32(P, A, R, b, k, kMassLo, kMassHi, S.w32, S.xa, S.xb, S.xs, s, fuse));
    bool x1 = false;
    if (df) {
        NM_TRY(launch_resid_df(R, A.nrows, A.rowptr.as<int>(), A.col.as<int>(), A.val32.as<float>(),
                               A.vlo32.as<float>(), W, ldw, S.xs, S.w32, b, s, P->use_vec, P->df_threads,
                               A.dinv32.as<float>(), it, fuse ? S.xa : nullptr));
        x1 = fuse;
    } else {
        NM_TRY(launch_resid_mixed(R, A.nrows, A.rowptr.as<int>(), A.col.as<int>(), A.val.as<double>(), W, ldw,
                                  S.xs, S.w32, b, s));
    }
    return cheb32(P, A, R, b, k, kMassLo, kMassHi, S.w32, S.xa, S.xb, S.es, s, x1);
}

// W = K_eff X in double with the pressure inverse by a refined solve.
static int apply_K_mixed_core(nm_problem* P, const double* X, int64_t ldx, double* W, int64_t ldw, int b,
                              int k_P, const MixScratch& S, cudaStream_t s, bool pre_split);

// ... and minus C^T S C X with self-gravitation.
static int apply_K_mixed(nm_problem* P, const double* X, int64_t ldx, double* W, int64_t ldw, int b, int k_P,
                         const MixScratch& S, cudaStream_t s, bool pre_split = false) {
    NM_TRY(apply_K_mixed_core(P, X, ldx, W, ldw, b, k_P, S, s, pre_split));
    return apply_selfgrav(P, X, ldx, W, ldw, b, s);
}

static int apply_K_mixed_core(nm_problem* P, const double* X, int64_t ldx, double* W, int64_t ldw, int b,
                              int k_P, const MixScratch& S, cudaStream_t s, bool pre_split) {
    Mats<double> m = mats<double>(P);
    const bool df = P->use_df != 0;
    // pre_split: S.Th / S.Tl already hold the exact float pair of X
    if (df && !pre_split) NM_TRY(launch_split(P->info.n, b, X, ldx, S.Th, S.Tl, s));
    Bsr33Args<double> a;
    a.nrows = (int)m.Nu;
    a.rowptr = m.u_rp;
    a.col = m.u_col;
    a.val = m.AG;
    a.b = b;
    a.X = X;
    a.ldx = ldx;
    a.W = W;
    a.ldw = ldw;
    // With "overlap", the pressure chain (E_G^T X, the refined A_p solve,
    // the combine) runs on the problem's high-priority aux stream while the
    // A_G product runs on s; E_G S is added after the join.
    const bool split_e = m.Np > 0 && P->overlap;
    cudaStream_t ps = s;
    if (split_e) {
        if (!P->aux) {
            int lo_pri = 0, hi_pri = 0;
            NM_CUDA(cudaDeviceGetStreamPriorityRange(&lo_pri, &hi_pri));
            NM_CUDA(cudaStreamCreateWithPriority(&P->aux, cudaStreamNonBlocking, hi_pri));
            NM_CUDA(cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming));
            NM_CUDA(cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming));
        }
        ps = P->aux;
        NM_CUDA(cudaEventRecord(P->ev_fork, s));
        NM_CUDA(cudaStreamWaitEvent(ps, P->ev_fork, 0));
    }
    if (m.Np > 0) {
        Bsr13Args<double> q;
        q.nrows = (int)m.Np;
        q.rowptr = m.et_rp;
        q.col = m.et_col;
        q.val = m.EGt;
        q.b = b;
        q.X = X;
        q.ldx = ldx;
        q.Q = S.Q64;
        q.ldq = b;
        NM_TRY(launch_bsr13<double>(q, ps));
        NM_TRY(mixed_solve(P, P->Pn, 1, b, k_P, S.Q64, b, S, P->use_df != 0, ps));
        CombineArgs c;
        c.rows = m.Np;
        c.b = b;
        c.x32 = S.xs;
        c.e32 = S.es;
        c.out = S.S64;
        NM_TRY(launch_combine(c, ps));
        if (!split_e) {
            a.e_rowptr = m.e_rp;
            a.e_col = m.e_col;
            a.e_val = m.EG;
            a.S = S.S64;
            a.lds = b;
        }
    }
    if (split_e) {
        NM_CUDA(cudaEventRecord(P->ev_join, ps));
        if (!df) {
            NM_TRY(launch_bsr33<double>(a, s));
        } else {
            Bsr33DfArgs f;
            f.nrows = a.nrows;
            f.rowptr = a.rowptr;
            f.col = a.col;
            f.vh = P->AG.val32.as<float>();
            f.vl = P->AG.vlo32.as<float>();
            f.Xh = S.Th;
            f.Xl = S.Tl;
            f.b = b;
            f.W = W;
            f.ldw = ldw;
            f.vec = P->use_vec;
            f.nt = P->df_threads;
            NM_TRY(launch_bsr33_df(f, s));
        }
        NM_CUDA(cudaStreamWaitEvent(s, P->ev_join, 0));
        return launch_bsr31_add((int)m.Nu, m.e_rp, m.e_col, m.EG, S.S64, b, b, W, ldw, s);
    }
    if (!df) return launch_bsr33<double>(a, s);
    Bsr33DfArgs f;
    f.nrows = a.nrows;
    f.rowptr = a.rowptr;
    f.col = a.col;
    f.vh = P->AG.val32.as<float>();
    f.vl = P->AG.vlo32.as<float>();
    f.Xh = S.Th;
    f.Xl = S.Tl;
    f.b = b;
    f.e_rowptr = a.e_rowptr;
    f.e_col = a.e_col;
    f.e_val = a.e_val;
    f.S = a.S;
    f.lds = a.lds;
    f.W = W;
    f.ldw = ldw;
    f.vec = P->use_vec;
    f.nt = P->df_threads;
    return launch_bsr33_df(f, s);
}

static int filter_apply_mixed(nm_problem* P, const nm_filter* f, const double* Y, int64_t ldy, double* Z,
                              int64_t ldz, int b, cudaStream_t s, const GammaTable* gt) {
    const int d = f->degree;
    if (d < 0 || (!f->gamma && !gt)) return fail(NM_EINVAL, "filter needs degree >= 0 and gamma");
    if (f->k_M < 1 || (P->info.Np > 0 && f->k_P < 1)) return fail(NM_EINVAL, "k_M and k_P must be >= 1");
    if (!(f->e > 0)) return fail(NM_EINVAL, "filter half-width e must be positive");
    if (f->m_lo > 0 || f->m_hi > 0) return fail(NM_EUNSUPPORTED, "mixed mode uses the P2 element bounds");
    NM_TRY(ensure_f32(P, s));
    if (P->use_df) NM_TRY(ensure_df(P, s));
    if (b == 32 && P->use_tma) NM_TRY(build_tma_tiles(P->Mr, s));
    const int64_t n = P->info.n;
    MixScratch S;
    NM_TRY(get_mix_scratch(P, b, S));
    if (gt) {
        for (int g = 0; g < gt->S; ++g)
            NM_TRY(launch_scale_copy<double>(n, gt->group, gt->host[g], Y + g * gt->group, ldy, Z + g * gt->group,
                                             ldz, s));
    } else {
        NM_TRY(launch_scale_copy<double>(n, b, f->gamma[0], Y, ldy, Z, ldz, s));
    }
    if (d == 0) return NM_OK;
    NM_TRY(launch_scale_copy<double>(n, b, 1.0, Y, ldy, S.TA, b, s));
    const int64_t kl = 1 + (P->info.Np > 0 ? 2 * f->k_P + 4 : 0);
    // One degree k of the recurrence (T_k in cur, T_{k-1} in prev; T_{k+1}
    // overwrites prev). With dev_gam the combine takes gamma_{k+1} from the
    // device table at the device-side degree counter (graph replay).
    auto degree = [&](int k, double* cur, double* prev, const double* dev_gam, int gstride, int ggroup,
                      const int* ctr) -> int {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        NM_TRY(prof_begin(P, s, &e0));
        NM_TRY(apply_K_mixed(P, cur, b, S.W, b, b, f->k_P, S, s, k > 0 && P->use_df));
        NM_TRY(prof_end(P, s, 1, e0, kl));
        NM_TRY(prof_begin(P, s, &e1));
        NM_TRY(mixed_solve(P, P->Mr, 3, b, f->k_M, S.W, b, S, P->use_df != 0, s));
        CombineArgs c;
        c.rows = n;
        c.b = b;
        c.x32 = S.xs;
        c.e32 = S.es;
        c.Tk = cur;
        c.Tp = k == 0 ? nullptr : prev;
        c.Tn = prev;
        c.Z = Z;
        c.ldz = ldz;
        c.a1 = (k == 0 ? 1.0 : 2.0) / f->e;
        c.cshift = f->c;
        c.a2 = k == 0 ? 0.0 : 1.0;
        if (dev_gam) {
            c.gam_tab = dev_gam;
            c.gam_stride = gstride;
            c.gam_group = ggroup;
            c.deg = ctr;
        } else {
            c.gam = gt ? 0.0 : f->gamma[k + 1];
            if (gt) {
                c.gam_tab = gt->dev + (int64_t)(k + 1) * gt->S;
                c.gam_group = gt->group;
            }
        }
        if (P->use_df && (dev_gam || k + 1 < d)) {   // the next degree's K_eff SpMM takes Tn split
            c.Th = S.Th;
            c.Tl = S.Tl;
        }
        NM_TRY(launch_combine(c, s));
        NM_TRY(prof_end(P, s, 0, e1, 2 * f->k_M + 3));
        return NM_OK;
    };
    const bool graphs = P->use_graphs && !P->profile && !P->overlap && s != nullptr && d >= 3;
    if (!graphs) {
        double* cur = S.TA;
        double* prev = S.TB;
        for (int k = 0; k < d; ++k) {
            NM_TRY(degree(k, cur, prev, nullptr, 0, 1, nullptr));
            std::swap(cur, prev);
        }
        return NM_OK;
    }
    // Graph replay of degrees 1..d-1 (the d x k_M launch chain): degree 0
    // runs eagerly; odd and even degrees differ only in which block holds
    // T_k, so two captured graphs serve them all, with gamma_{k+1} read
    // from a device table at a device-side degree counter that each graph
    // advances at its end.
    NM_TRY(degree(0, S.TA, S.TB, nullptr, 0, 1, nullptr));
    const double* gtab;
    int gstride, ggroup;
    if (gt) {
        gtab = gt->dev;
        gstride = gt->S;
        ggroup = gt->group;
    } else {
        const size_t gbytes = (size_t)(d + 1) * sizeof(double);
        if (P->graph_gam.bytes < gbytes) NM_TRY(P->graph_gam.alloc(gbytes));
        NM_CUDA(cudaMemcpyAsync(P->graph_gam.p, f->gamma, gbytes, cudaMemcpyHostToDevice, s));
        gtab = P->graph_gam.as<double>();
        gstride = 1;
        ggroup = b;
    }
    if (!P->graph_deg.p) NM_TRY(P->graph_deg.alloc(sizeof(int)));
    int* ctr = P->graph_deg.as<int>();
    NM_TRY(launch_set_int(ctr, 1, s));
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    uint64_t nodes[2] = {0, 0};
    auto drop = [&]() {
        for (auto& x : exec)
            if (x) cudaGraphExecDestroy(x);
    };
    for (int par = 0; par < 2; ++par) {   // par 0: odd degrees (T_k in TB), par 1: even
        double* cur = par == 0 ? S.TB : S.TA;
        double* prev = par == 0 ? S.TA : S.TB;
        const uint64_t l0 = launches_so_far();
        NM_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        int rc = degree(par == 0 ? 1 : 2, cur, prev, gtab, gstride, ggroup, ctr);
        if (rc == NM_OK) rc = launch_inc_int(ctr, s);
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(s, &g);
        nodes[par] = launches_so_far() - l0;
        count_launch((uint64_t)0 - nodes[par]);   // captured, not launched
        if (rc != NM_OK || ec != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            drop();
            cudaGetLastError();
            return rc != NM_OK ? rc : fail(NM_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
        }
        const cudaError_t ei = cudaGraphInstantiate(&exec[par], g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            drop();
            return fail(NM_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ei));
        }
    }
    for (int k = 1; k < d; ++k) {
        const int par = (k & 1) ? 0 : 1;
        const cudaError_t el = cudaGraphLaunch(exec[par], s);
        if (el != cudaSuccess) {
            drop();
            return fail(NM_ECUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(el));
        }
        count_launch(nodes[par]);
    }
    drop();   // released once the launched graphs complete
    return NM_OK;
}

int filter_apply_mixed_pub(nm_problem* P, const nm_filter* f, const double* Y, int64_t ldy, double* Z, int64_t ldz,
                           int b, cudaStream_t s) {
    return filter_apply_mixed(P, f, Y, ldy, Z, ldz, b, s);
}

int apply_K_mixed_pub(nm_problem* P, const double* X, int64_t ldx, double* Y, int64_t ldy, int b, int k_P,
                      cudaStream_t s) {
    NM_TRY(ensure_f32(P, s));
    if (P->use_df) NM_TRY(ensure_df(P, s));
    MixScratch S;
    NM_TRY(get_mix_scratch(P, b, S));
    return apply_K_mixed(P, X, ldx, Y, ldy, b, k_P, S, s);
}

int solve_M_mixed_pub(nm_problem* P, int k_M, const double* W, int64_t ldw, double* X, int64_t ldx, int b,
                      cudaStream_t s) {
    NM_TRY(ensure_f32(P, s));
    if (P->use_df) NM_TRY(ensure_df(P, s));
    if (b == 32 && P->use_tma) NM_TRY(build_tma_tiles(P->Mr, s));
    MixScratch S;
    NM_TRY(get_mix_scratch(P, b, S));
    NM_TRY(mixed_solve(P, P->Mr, 3, b, k_M, W, ldw, S, P->use_df != 0, s));
    CombineArgs c;
    c.rows = P->info.n;
    c.b = b;
    c.x32 = S.xs;
    c.e32 = S.es;
    c.out = S.W;
    NM_TRY(launch_combine(c, s));
    return launch_scale_copy<double>(P->info.n, b, 1.0, S.W, b, X, ldx, s);
}

// ------------------------------------------------------------------ profiling
int prof_begin(nm_problem* P, cudaStream_t s, cudaEvent_t* start) {
    *start = nullptr;
    if (!P->profile) return NM_OK;
    if (P->ev_next + 2 > P->ev_pool.size()) {
        for (int i = 0; i < 256; ++i) {
            cudaEvent_t e;
            NM_CUDA(cudaEventCreate(&e));
            P->ev_pool.push_back(e);
        }
    }
    *start = P->ev_pool[P->ev_next++];
    NM_CUDA(cudaEventRecord(*start, s));
    return NM_OK;
}

int prof_end(nm_problem* P, cudaStream_t s, int kind, cudaEvent_t start, int64_t launches) {
    if (!P->profile || !start) return NM_OK;
    cudaEvent_t stop = P->ev_pool[P->ev_next++];
    NM_CUDA(cudaEventRecord(stop, s));
    P->ev_regions.push_back({kind, {start, stop}});
    P->ev_launches.push_back(launches);
    return NM_OK;
}

int profile_read(nm_problem* P, int kind, int64_t* launches, double* ms) {
    int64_t l = 0;
    double t = 0.0;
    for (size_t i = 0; i < P->ev_regions.size(); ++i) {
        if (P->ev_regions[i].first != kind) continue;
        NM_CUDA(cudaEventSynchronize(P->ev_regions[i].second.second));
        float x = 0.f;
        NM_CUDA(cudaEventElapsedTime(&x, P->ev_regions[i].second.first, P->ev_regions[i].second.second));
        t += x;
        l += P->ev_launches[i];
    }
    *launches = l;
    *ms = t;
    return NM_OK;
}

int profile_set(nm_problem* P, int enable, int reset) {
    if (reset || !enable) {
        // fold nothing: a reset discards the recorded regions (events are reused)
        for (auto& r : P->ev_regions) {
            cudaEventSynchronize(r.second.second);
        }
        P->ev_regions.clear();
        P->ev_launches.clear();
        P->ev_next = 0;
    }
    P->profile = enable;
    return NM_OK;
}

template <typename T>
int filter_apply_t(nm_problem* P, const nm_filter* f, const T* Y, int64_t ldy, T* Z, int64_t ldz, int b,
                   cudaStream_t s) {
    return filter_core<T>(P, f, Y, ldy, Z, ldz, b, nullptr, s);
}

// ------------------------------------------------------------------ public pieces
template <typename T>
int apply_K_pub(nm_problem* P, const T* X, int64_t ldx, T* Y, int64_t ldy, int b, int k_P, cudaStream_t s) {
    Scratch<T> S;
    NM_TRY(get_scratch<T>(P, b, S));
    return apply_K_t<T>(P, X, ldx, Y, ldy, b, k_P, S, nullptr, 0.0, s);
}

template <typename T>
int apply_M_pub(nm_problem* P, const T* X, int64_t ldx, T* Y, int64_t ldy, int b, int mode,
                const double* sk, cudaStream_t s) {
    Mats<T> m = mats<T>(P);
    KronArgs<T> a;
    a.nrows = (int)m.Nu;
    a.rowptr = m.u_rp;
    a.col = m.u_col;
    a.val = m.Mr;
    a.b = b;
    a.X = X;
    a.ldx = ldx;
    a.Y = Y;
    a.ldy = ldy;
    if (sk)
        for (int i = 0; i < 9; ++i) a.sk[i] = (T)sk[i];
    return launch_kron<T>(3, mode, a, s);
}

template <typename T>
__global__ void dscale_kernel(int64_t Nu, int b, T inv_theta, const T* dinv, const T* W, int64_t ldw,
                              T* X, int64_t ldx) {
    const int64_t total = 3 * Nu * b;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / b;
        const int c = (int)(t - r * b);
        X[r * ldx + c] = inv_theta * dinv[r / 3] * W[r * ldw + c];
    }
}

template <typename T>
int solve_M_pub(nm_problem* P, int k_M, double lo, double hi, const T* W, int64_t ldw, T* X,
                int64_t ldx, int b, cudaStream_t s) {
    if (k_M < 1) return fail(NM_EINVAL, "k_M must be >= 1");
    const double mlo = lo > 0 ? lo : kMassLo, mhi = hi > 0 ? hi : kMassHi;
    if (!(mhi > mlo)) return fail(NM_EINVAL, "mass bounds need hi > lo > 0");
    Scratch<T> S;
    NM_TRY(get_scratch<T>(P, b, S));
    Mats<T> m = mats<T>(P);
    const ChebCoef cc(mlo, mhi);
    const int64_t n = P->info.n;
    int64_t g = (n * b + 255) / 256;
    if (g > 4864) g = 4864;
    if (k_M == 1) {
        dscale_kernel<T><<<(unsigned)g, 256, 0, s>>>(m.Nu, b, (T)cc.inv_theta, m.dM, W, ldw, X, ldx);
        count_launch();
        NM_CUDA(cudaGetLastError());
        return NM_OK;
    }
    // W is the right-hand side of every step: copy it into the scratch slot
    NM_TRY(launch_scale_copy<T>(n, b, (T)1, W, ldw, S.W, b, s));
    dscale_kernel<T><<<(unsigned)g, 256, 0, s>>>(m.Nu, b, (T)cc.inv_theta, m.dM, S.W, b, S.XA, b);
    count_launch();
        NM_CUDA(cudaGetLastError());
    return mass_steps<T>(m, b, k_M, mlo, mhi, S, nullptr, nullptr, nullptr, nullptr, nullptr, 0, X, ldx, s);
}

// ------------------------------------------------------------------ caller-supplied scratch
// Bytes of scratch the FP64 filter recurrence uses for b columns: five n x b
// blocks (T_k, T_{k-1}, K_eff T_k, two mass-solve iterates) and three Np x b
// blocks (E_G^T X and two pressure iterates), the layout get_scratch uses.
size_t filter_scratch_bytes(const nm_problem* P, int b) {
    return (size_t)(5 * P->info.n + 3 * P->info.Np) * (size_t)b * sizeof(double);
}

// The FP64 filter recurrence of Sec. 5 (Z = sum_k gamma_k T_k(B) Y) on
// scratch the caller hands in: at least filter_scratch_bytes(P, b) bytes,
// 256-byte aligned. Performs no device allocation and records no profile
// regions; launches the same kernels in the same order as the FP64 branch
// of nm_filter_apply.
int filter_apply_on(nm_problem* P, const nm_filter* f, const double* Y, int64_t ldy, double* Z, int64_t ldz,
                    int b, double* scratch, cudaStream_t s) {
    const int d = f->degree;
    if (d < 0 || !f->gamma) return fail(NM_EINVAL, "filter needs degree >= 0 and gamma");
    if (f->k_M < 2 || (P->info.Np > 0 && f->k_P < 2)) return fail(NM_EINVAL, "k_M and k_P must be >= 2");
    if (!(f->e > 0)) return fail(NM_EINVAL, "filter half-width e must be positive");
    const double mlo = f->m_lo > 0 ? f->m_lo : kMassLo;
    const double mhi = f->m_hi > 0 ? f->m_hi : kMassHi;
    if (!(mhi > mlo)) return fail(NM_EINVAL, "mass bounds need m_hi > m_lo > 0");
    const int64_t n = P->info.n, Np = P->info.Np;
    Scratch<double> S;
    double* p = scratch;
    S.TA = p; p += n * b;
    S.TB = p; p += n * b;
    S.W = p; p += n * b;
    S.XA = p; p += n * b;
    S.XB = p; p += n * b;
    S.Q = p; p += Np * b;
    S.PA = p; p += Np * b;
    S.PB = p;
    Mats<double> m = mats<double>(P);
    const ChebCoef cc(mlo, mhi);
    NM_TRY(launch_scale_copy<double>(n, b, f->gamma[0], Y, ldy, Z, ldz, s));
    if (d == 0) return NM_OK;
    NM_TRY(launch_scale_copy<double>(n, b, 1.0, Y, ldy, S.TA, b, s));
    double* cur = S.TA;   // T_k
    double* prev = S.TB;  // T_{k-1}, overwritten by T_{k+1}
    for (int k = 0; k < d; ++k) {
        NM_TRY(apply_K_t<double>(P, cur, b, S.W, b, b, f->k_P, S, S.XA, cc.inv_theta, s));
        FiltStep fs;
        fs.cshift = f->c;
        fs.gam = f->gamma[k + 1];
        fs.a1 = (k == 0 ? 1.0 : 2.0) / f->e;
        fs.a2 = k == 0 ? 0.0 : 1.0;
        NM_TRY(mass_steps<double>(m, b, f->k_M, mlo, mhi, S, &fs, cur, k == 0 ? nullptr : prev, prev, Z, ldz,
                                  nullptr, 0, s));
        std::swap(cur, prev);
    }
    return NM_OK;
}

template int filter_apply_t<double>(nm_problem*, const nm_filter*, const double*, int64_t, double*, int64_t, int, cudaStream_t);
template int filter_apply_t<float>(nm_problem*, const nm_filter*, const float*, int64_t, float*, int64_t, int, cudaStream_t);
template int apply_K_pub<double>(nm_problem*, const double*, int64_t, double*, int64_t, int, int, cudaStream_t);
template int apply_K_pub<float>(nm_problem*, const float*, int64_t, float*, int64_t, int, int, cudaStream_t);
template int apply_M_pub<double>(nm_problem*, const double*, int64_t, double*, int64_t, int, int, const double*, cudaStream_t);
template int apply_M_pub<float>(nm_problem*, const float*, int64_t, float*, int64_t, int, int, const double*, cudaStream_t);
template int solve_M_pub<double>(nm_problem*, int, double, double, const double*, int64_t, double*, int64_t, int, cudaStream_t);
template int solve_M_pub<float>(nm_problem*, int, double, double, const float*, int64_t, float*, int64_t, int, cudaStream_t);

// ------------------------------------------------------------------ autotuner
int set_tile_rows(nm_problem* P, int64_t rows);

// Device milliseconds of `reps` filter degrees (one filter_apply of degree
// reps) on the problem's stream.
static int time_degree(nm_problem* P, int b, nm_prec prec, int k_M, const void* Y, void* Z, int reps, double* ms) {
    cudaStream_t s = P->ctx->stream;
    std::vector<double> gamma(reps + 1, 0.5);
    const double lo = -1.0, hi = 2.0 * (P->bounds_hi > 0 ? P->bounds_hi : 1.0);
    nm_filter f{reps, gamma.data(), 0.5 * (hi + lo), 0.5 * (hi - lo), k_M, k_M, 0.0, 0.0};
    auto run = [&]() -> int {
        if (prec == NM_F64) return filter_apply_t<double>(P, &f, (const double*)Y, b, (double*)Z, b, b, s);
        if (prec == NM_F32) return filter_apply_t<float>(P, &f, (const float*)Y, b, (float*)Z, b, b, s);
        return filter_apply_mixed(P, &f, (const double*)Y, b, (double*)Z, b, b, s);
    };
    NM_TRY(run());   // warm-up (also allocates the scratch)
    cudaEvent_t e0, e1;
    NM_CUDA(cudaEventCreate(&e0));
    NM_CUDA(cudaEventCreate(&e1));
    NM_CUDA(cudaEventRecord(e0, s));
    int rc = run();
    NM_CUDA(cudaEventRecord(e1, s));
    NM_CUDA(cudaEventSynchronize(e1));
    float x = 0.f;
    cudaEventElapsedTime(&x, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = x;
    return rc;
}

int autotune(nm_problem* P, int b, nm_prec prec, int k_M, std::string* report) {
    if (b < 1 || b > 64) return fail(NM_EINVAL, "block width must be in 1..64");
    if (k_M < 2) k_M = prec == NM_F64 ? 38 : (prec == NM_MIXED ? 20 : 28);
    cudaStream_t s = P->ctx->stream;
    if (prec != NM_F64) NM_TRY(ensure_f32(P, s));
    if (prec == NM_MIXED) NM_TRY(ensure_df(P, s));
    const int64_t n = P->info.n;
    const size_t es = prec == NM_F32 ? sizeof(float) : sizeof(double);
    DevBuf Y, Z;
    NM_TRY(Y.alloc((size_t)n * 64 * es));
    NM_TRY(Z.alloc((size_t)n * 64 * es));
    NM_CUDA(cudaMemsetAsync(Y.p, 0, (size_t)n * 64 * es, s));
    if (prec == NM_F32) {
        // float start block: 64 columns of Gaussians drawn in double and narrowed
        NM_TRY(launch_philox_normal(n * 32, 7, Z.as<double>(), s));
        NM_TRY((launch_convert<double, float>(n, 32, Z.as<double>(), 32, Y.as<float>(), 32, s)));
        NM_TRY((launch_convert<double, float>(n, 32, Z.as<double>(), 32, Y.as<float>() + n * 32, 32, s)));
    } else {
        NM_TRY(launch_philox_normal(n * 64, 7, Y.as<double>(), s));
    }
    struct Cfg { int sched, tile, tk, df, chunk, vec, graphs, tma; };
    std::vector<Cfg> cfgs;
    const int df1 = prec == NM_MIXED ? 1 : P->use_df;
    for (int sched : {0, 1})
        for (int df : (prec == NM_MIXED ? std::vector<int>{1, 0} : std::vector<int>{P->use_df}))
            cfgs.push_back({sched, 0, 2, df, 0, 1, 0, 0});
    if (prec == NM_MIXED) cfgs.push_back({0, 0, 2, 1, 0, 1, 1, 0});
    if (prec == NM_MIXED && b == 32) cfgs.push_back({0, 0, 2, 1, 0, 1, 0, 1});
    if (prec != NM_F64 && b == 32) cfgs.push_back({0, 0, 2, df1, 0, 0, 0, 0});
    if (b >= 17)
        for (int ch : {256, 512, 1024}) cfgs.push_back({0, 0, 2, df1, ch, 0, 0, 0});
    if (prec != NM_F64 && b == 32) {
        cfgs.push_back({0, 16, 2, df1, 0, 0, 0, 0});
        cfgs.push_back({0, 32, 2, df1, 0, 0, 0, 0});
    }
    const int reps = 6;   // degrees per timing (graph replay needs at least 3)
    double best = 1e300;
    Cfg bestc = cfgs[0];
    std::string rep = "{\"b\": " + std::to_string(b) + ", \"variants\": [";
    for (size_t i = 0; i < cfgs.size(); ++i) {
        const Cfg& c = cfgs[i];
        P->use_sched = c.sched;
        P->use_df = c.df;
        P->use_chunk = c.chunk;
        P->use_vec = c.vec;
        P->use_graphs = c.graphs;
        P->use_tma = c.tma;
        NM_TRY(set_tile_rows(P, c.tile));
        if (c.tile) P->Mr.tile_kernel = P->Pn.tile_kernel = c.tk;
        double ms = 0;
        NM_TRY(time_degree(P, b, prec, k_M, Y.p, Z.p, reps, &ms));
        ms /= reps;
        char buf[192];
        snprintf(buf, sizeof buf,
                 "%s{\"sched\": %d, \"chunk\": %d, \"vec\": %d, \"graphs\": %d, \"tma\": %d, \"tile_rows\": %d, "
                 "\"double_float\": %d, \"ms_per_degree\": %.4f}",
                 i ? ", " : "", c.sched, c.chunk, c.vec, c.graphs, c.tma, c.tile, c.df, ms);
        rep += buf;
        if (ms < best) {
            best = ms;
            bestc = c;
        }
    }
    P->use_sched = bestc.sched;
    P->use_df = bestc.df;
    P->use_chunk = bestc.chunk;
    P->use_vec = bestc.vec;
    P->use_graphs = bestc.graphs;
    P->use_tma = bestc.tma;
    NM_TRY(set_tile_rows(P, bestc.tile));
    if (bestc.tile) P->Mr.tile_kernel = P->Pn.tile_kernel = bestc.tk;
    rep += "], \"chosen\": {\"sched\": " + std::to_string(bestc.sched) + ", \"chunk\": " +
           std::to_string(bestc.chunk) + ", \"vec\": " + std::to_string(bestc.vec) + ", \"graphs\": " +
           std::to_string(bestc.graphs) + ", \"tma\": " + std::to_string(bestc.tma) + ", \"tile_rows\": " +
           std::to_string(bestc.tile) + ", \"double_float\": " + std::to_string(bestc.df) + "}, \"us_per_column_degree\": {";
    int first = 1;
    for (int bb : {16, 32, 64}) {
        double ms = 0;
        NM_TRY(time_degree(P, bb, prec, k_M, Y.p, Z.p, reps, &ms));
        char buf[64];
        snprintf(buf, sizeof buf, "%s\"%d\": %.3f", first ? "" : ", ", bb, 1e3 * ms / reps / bb);
        rep += buf;
        first = 0;
    }
    rep += "}}";
    *report = rep;
    return NM_OK;
}

// ------------------------------------------------------------------ filter design
void jackson_step_coeffs(double lam_lo, double lam_hi, double xi, double eta, int d, double* gamma,
                         double* c, double* e) {
    *c = 0.5 * (lam_hi + lam_lo);
    *e = 0.5 * (lam_hi - lam_lo);
    double al = (xi - *c) / *e, be = (eta - *c) / *e;
    al = std::min(1.0, std::max(-1.0, al));
    be = std::min(1.0, std::max(-1.0, be));
    const double ta = std::acos(al), tb = std::acos(be);
    const double ad = M_PI / (d + 2);
    for (int k = 0; k <= d; ++k) {
        const double mu = k == 0 ? (ta - tb) / M_PI : 2.0 * (std::sin(k * ta) - std::sin(k * tb)) / (k * M_PI);
        const double g = ((1.0 - (double)k / (d + 2)) * std::sin(ad) * std::cos(k * ad) +
                          std::cos(ad) * std::sin(k * ad) / (d + 2)) / std::sin(ad);
        gamma[k] = g * mu;
    }
}

static double cheb_sum(const std::vector<double>& g, double t) {
    t = std::min(1.0, std::max(-1.0, t));
    double T0 = 1, T1 = t, s = g[0];
    if (g.size() > 1) s += g[1] * T1;
    for (size_t k = 2; k < g.size(); ++k) {
        const double T2 = 2 * t * T1 - T0;
        s += g[k] * T2;
        T0 = T1;
        T1 = T2;
    }
    return s;
}

// ------------------------------------------------------------------ dense helpers
struct Dense {
    nm_ctx* ctx;
    cudaStream_t s;
};

// C (m x b, col-major) = V^T (M W) + beta C: V row-major n x m (ld ldv),
// MW row-major n x b (ld ldw). By default the FP64-accurate tensor-core
// product (ozaki_gemm.cu); option "dense_tc" = 0 uses cuBLAS DGEMM.
static int gemm_VtW(nm_ctx* ctx, int64_t n, int m, int b, const double* V, int64_t ldv,
                    const double* MW, int64_t ldw, double* C, double beta) {
    if (ctx->dense_tc) return ozaki_gemm_tn(ctx, ctx->stream, m, b, n, 1.0, V, ldv, MW, ldw, beta, C, m);
    const double one = 1.0;
    NM_CUBLAS(cublasDgemm(ctx->cublas, CUBLAS_OP_N, CUBLAS_OP_T, m, b, (int)n, &one, V, (int)ldv, MW,
                          (int)ldw, &beta, C, m));
    return NM_OK;
}

// W (row-major n x b, ld ldw) += alpha * V C, C col-major m x b
static int gemm_WmVC(nm_ctx* ctx, int64_t n, int m, int b, double alpha, const double* V, int64_t ldv,
                     const double* C, int ldc, double* W, int64_t ldw) {
    if (ctx->dense_tc) return ozaki_gemm_nn(ctx->stream, n, b, m, alpha, V, ldv, C, ldc, 1.0, W, ldw);
    const double one = 1.0;
    NM_CUBLAS(cublasDgemm(ctx->cublas, CUBLAS_OP_T, CUBLAS_OP_N, b, (int)n, m, &alpha, C, ldc, V,
                          (int)ldv, &one, W, (int)ldw));
    return NM_OK;
}

// X (row-major n x k, ld ldx) = V S with V row-major n x m (ld ldv) and S
// col-major m x k (ld lds).
static int gemm_VS(nm_ctx* ctx, int64_t n, int m, int k, const double* V, int64_t ldv, const double* S, int lds,
                   double* X, int64_t ldx) {
    if (ctx->dense_tc) return ozaki_gemm_nn(ctx->stream, n, k, m, 1.0, V, ldv, S, lds, 0.0, X, ldx);
    const double one = 1.0, zero = 0.0;
    NM_CUBLAS(cublasDgemm(ctx->cublas, CUBLAS_OP_T, CUBLAS_OP_N, k, (int)n, m, &one, S, lds, V, (int)ldv, &zero, X,
                          (int)ldx));
    return NM_OK;
}

template <typename T>
struct OpBuf {
    DevBuf f_in, f_out;   // float staging for the FP32 filter
};

// W = p(B) V_j (prec selects the filter arithmetic); V_j, W FP64 row-major
static int filter_block(nm_problem* P, nm_prec prec, int d, double c, double e, int k_M, int k_P, const double* Y,
                        int64_t ldy, double* W, int64_t ldw, const GammaTable* gt, DevBuf& fin, DevBuf& fout,
                        cudaStream_t s) {
    const int64_t n = P->info.n;
    const int b = gt->S * gt->group;
    nm_filter f{d, nullptr, c, e, k_M, k_P, 0.0, 0.0};
    if (prec == NM_F64) return filter_core<double>(P, &f, Y, ldy, W, ldw, b, gt, s);
    if (prec == NM_MIXED) return filter_apply_mixed(P, &f, Y, ldy, W, ldw, b, s, gt);
    NM_TRY(ensure_f32(P, s));
    if (fin.bytes < (size_t)n * b * sizeof(float)) {
        fin.release();
        fout.release();
        NM_TRY(fin.alloc((size_t)n * b * sizeof(float)));
        NM_TRY(fout.alloc((size_t)n * b * sizeof(float)));
    }
    NM_TRY((launch_convert<double, float>(n, b, Y, ldy, fin.as<float>(), b, s)));
    NM_TRY(filter_core<float>(P, &f, fin.as<float>(), b, fout.as<float>(), b, b, gt, s));
    return launch_convert<float, double>(n, b, fout.as<float>(), b, W, ldw, s);
}

// Apply K_eff (FP64, effectively exact Schur term) or M to m columns of a
// row-major n x m block in chunks of <= 64 columns.
static int apply_cols(nm_problem* P, int which, const double* V, int64_t ldv, double* Y, int64_t ldy,
                      int m, int k_P, cudaStream_t s) {
    for (int c0 = 0; c0 < m; c0 += 64) {
        const int bc = std::min(64, m - c0);
        if (which == 0)
            NM_TRY(apply_K_pub<double>(P, V + c0, ldv, Y + c0, ldy, bc, k_P, s));
        else if (which == 1)
            NM_TRY(apply_M_pub<double>(P, V + c0, ldv, Y + c0, ldy, bc, KRON_PLAIN, nullptr, s));
        else {
            const double* O = P->Omega;
            const double sk[9] = {0, -O[2], O[1], O[2], 0, -O[0], -O[1], O[0], 0};
            NM_TRY(apply_M_pub<double>(P, V + c0, ldv, Y + c0, ldy, bc, KRON_CORI, sk, s));
        }
    }
    return NM_OK;
}

// Symmetric dense eigensolve on the device: A (m x m col-major, overwritten by
// eigenvectors), w (m). With B != nullptr the generalized problem A x = w B x.
static int dense_eig(nm_ctx* ctx, int m, double* A, double* B, double* w) {
    int lwork = 0;
    DevBuf info;
    NM_TRY(info.alloc(sizeof(int)));
    if (B) {
        NM_CUSOLVER(cusolverDnDsygvd_bufferSize(ctx->cusolver, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR,
                                                CUBLAS_FILL_MODE_UPPER, m, A, m, B, m, w, &lwork));
        DevBuf work;
        NM_TRY(work.alloc(std::max(lwork, 1) * sizeof(double)));
        NM_CUSOLVER(cusolverDnDsygvd(ctx->cusolver, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR,
                                     CUBLAS_FILL_MODE_UPPER, m, A, m, B, m, w, work.as<double>(), lwork,
                                     info.as<int>()));
    } else {
        NM_CUSOLVER(cusolverDnDsyevd_bufferSize(ctx->cusolver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER,
                                                m, A, m, w, &lwork));
        DevBuf work;
        NM_TRY(work.alloc(std::max(lwork, 1) * sizeof(double)));
        NM_CUSOLVER(cusolverDnDsyevd(ctx->cusolver, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, m, A, m,
                                     w, work.as<double>(), lwork, info.as<int>()));
    }
    int h = 0;
    NM_CUDA(cudaMemcpyAsync(&h, info.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    NM_CUDA(cudaStreamSynchronize(ctx->stream));
    if (h != 0) return fail(NM_ENOTCONV, "dense eigensolver failed, info = " + std::to_string(h));
    return NM_OK;
}

__global__ void symmetrize_kernel(int m, double* A) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i < m && j < i) {
        const double v = 0.5 * (A[i + (int64_t)j * m] + A[j + (int64_t)i * m]);
        A[i + (int64_t)j * m] = v;
        A[j + (int64_t)i * m] = v;
    }
}

static int symmetrize(int m, double* A, cudaStream_t s) {
    dim3 g((m + 127) / 128, m);
    symmetrize_kernel<<<g, 128, 0, s>>>(m, A);
    count_launch();
        NM_CUDA(cudaGetLastError());
    return NM_OK;
}

// M-orthonormalise W (row-major n x b) in place with Cholesky-QR; R (b x b col-major upper) out.
static int m_orth(nm_problem* P, double* W, int64_t ldw, int b, double* MW, double* G, int* rank_ok,
                  cudaStream_t s) {
    nm_ctx* ctx = P->ctx;
    const int64_t n = P->info.n;
    NM_TRY(apply_M_pub<double>(P, W, ldw, MW, b, b, KRON_PLAIN, nullptr, s));
    NM_TRY(gemm_VtW(ctx, n, b, b, W, ldw, MW, b, G, 0.0));
    NM_TRY(symmetrize(b, G, s));
    int lwork = 0;
    NM_CUSOLVER(cusolverDnDpotrf_bufferSize(ctx->cusolver, CUBLAS_FILL_MODE_UPPER, b, G, b, &lwork));
    DevBuf work, info;
    NM_TRY(work.alloc(std::max(lwork, 1) * sizeof(double)));
    NM_TRY(info.alloc(sizeof(int)));
    NM_CUSOLVER(cusolverDnDpotrf(ctx->cusolver, CUBLAS_FILL_MODE_UPPER, b, G, b, work.as<double>(), lwork,
                                 info.as<int>()));
    int h = 0;
    NM_CUDA(cudaMemcpyAsync(&h, info.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    NM_CUDA(cudaStreamSynchronize(s));
    *rank_ok = h == 0;
    if (h != 0) return NM_OK;
    // W <- W R^{-1}: in column-major terms Wc (b x n) <- R^{-T} Wc
    const double one = 1.0;
    NM_CUBLAS(cublasDtrsm(ctx->cublas, CUBLAS_SIDE_LEFT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_T,
                          CUBLAS_DIAG_NON_UNIT, b, (int)n, &one, G, b, W, (int)ldw));
    return NM_OK;
}

struct RRResult {
    std::vector<double> lam, res;
    int i0 = 0, k = 0;
};

// Rayleigh-Ritz of (K_eff, M) on V (n x m row-major, ld ldv, FP64). If X is
// non-null the selected Ritz vectors are written there (n x k, ld k).
// With sw (host, m x nw column-major: orthonormal coefficients of the
// converged wanted Ritz vectors of p(B)) a Ritz pair inside the slice is
// kept only if at least half of its coefficient vector lies in their span.
// The others are spurious Ritz values of the whole basis: mixtures of
// unconverged directions from both sides of the slice (seen with the
// self-gravitating planet, whose spectrum has eigenvalues far below and far
// above the slice at the same filter value).
static int rayleigh_ritz(nm_problem* P, const double* V, int64_t ldv, int m, double lam_lo, double lam_hi,
                         DevBuf* X, RRResult& out, const double* sw = nullptr, int nw = 0) {
    nm_ctx* ctx = P->ctx;
    cudaStream_t s = ctx->stream;
    const int64_t n = P->info.n;
    DevBuf KV, MV, H, G, w;
    NM_TRY(KV.alloc((size_t)n * m * sizeof(double)));
    NM_TRY(MV.alloc((size_t)n * m * sizeof(double)));
    NM_TRY(H.alloc((size_t)m * m * sizeof(double)));
    NM_TRY(G.alloc((size_t)m * m * sizeof(double)));
    NM_TRY(w.alloc((size_t)m * sizeof(double)));
    NM_TRY(apply_cols(P, 0, V, ldv, KV.as<double>(), m, m, 80, s));
    NM_TRY(apply_cols(P, 1, V, ldv, MV.as<double>(), m, m, 0, s));
    NM_TRY(gemm_VtW(ctx, n, m, m, V, ldv, KV.as<double>(), m, H.as<double>(), 0.0));
    NM_TRY(gemm_VtW(ctx, n, m, m, V, ldv, MV.as<double>(), m, G.as<double>(), 0.0));
    NM_TRY(symmetrize(m, H.as<double>(), s));
    NM_TRY(symmetrize(m, G.as<double>(), s));
    NM_TRY(dense_eig(ctx, m, H.as<double>(), G.as<double>(), w.as<double>()));
    std::vector<double> hw(m);
    NM_CUDA(cudaMemcpyAsync(hw.data(), w.p, m * sizeof(double), cudaMemcpyDeviceToHost, s));
    NM_CUDA(cudaStreamSynchronize(s));
    int i0 = 0;
    while (i0 < m && hw[i0] < lam_lo) ++i0;
    int i1 = i0;
    while (i1 < m && hw[i1] <= lam_hi) ++i1;
    int k = i1 - i0;
    out.i0 = i0;
    const double* Ssel = H.as<double>() + (int64_t)i0 * m;   // eigenvectors, col-major m x m
    DevBuf Skeep;
    out.lam.clear();
    if (sw && nw > 0 && k > 0) {
        std::vector<double> hz((size_t)m * k);
        NM_CUDA(cudaMemcpy(hz.data(), Ssel, hz.size() * sizeof(double), cudaMemcpyDeviceToHost));
        std::vector<int> keep;
        for (int j = 0; j < k; ++j) {
            const double* z = hz.data() + (size_t)j * m;
            double zz = 0, pp = 0;
            for (int r = 0; r < m; ++r) zz += z[r] * z[r];
            for (int c = 0; c < nw; ++c) {
                double d = 0;
                for (int r = 0; r < m; ++r) d += sw[(size_t)c * m + r] * z[r];
                pp += d * d;
            }
            if (pp >= 0.5 * zz) keep.push_back(j);
        }
        if ((int)keep.size() < k) {
            std::vector<double> hk((size_t)m * keep.size());
            for (size_t q = 0; q < keep.size(); ++q) {
                std::copy(hz.begin() + (size_t)keep[q] * m, hz.begin() + (size_t)(keep[q] + 1) * m,
                          hk.begin() + q * m);
                out.lam.push_back(hw[i0 + keep[q]]);
            }
            k = (int)keep.size();
            if (k > 0) {
                NM_TRY(Skeep.alloc(hk.size() * sizeof(double)));
                NM_CUDA(cudaMemcpy(Skeep.p, hk.data(), hk.size() * sizeof(double), cudaMemcpyHostToDevice));
                Ssel = Skeep.as<double>();
            }
        }
    }
    if (out.lam.empty()) out.lam.assign(hw.begin() + i0, hw.begin() + i0 + k);
    out.k = k;
    out.res.assign(k, 0.0);
    if (k == 0) return NM_OK;
    DevBuf KX, MX, lam_d, nr, nm_;
    NM_TRY(KX.alloc((size_t)n * k * sizeof(double)));
    NM_TRY(MX.alloc((size_t)n * k * sizeof(double)));
    NM_TRY(lam_d.alloc(k * sizeof(double)));
    NM_TRY(nr.alloc(k * sizeof(double)));
    NM_TRY(nm_.alloc(k * sizeof(double)));
    // X (n x k) = V S_sel
    auto proj = [&](const double* Vsrc, int64_t ld, double* dst) -> int {
        return gemm_VS(ctx, n, m, k, Vsrc, ld, Ssel, m, dst, k);
    };
    NM_TRY(proj(KV.as<double>(), m, KX.as<double>()));
    NM_TRY(proj(MV.as<double>(), m, MX.as<double>()));
    NM_CUDA(cudaMemcpyAsync(lam_d.p, out.lam.data(), k * sizeof(double), cudaMemcpyHostToDevice, s));
    NM_TRY(launch_resid_block(n, k, KX.as<double>(), MX.as<double>(), lam_d.as<double>(), KX.as<double>(), s));
    NM_CUDA(cudaMemsetAsync(nr.p, 0, k * sizeof(double), s));
    NM_CUDA(cudaMemsetAsync(nm_.p, 0, k * sizeof(double), s));
    NM_TRY(launch_colnorm2(n, k, KX.as<double>(), k, nr.as<double>(), s));
    NM_TRY(launch_colnorm2(n, k, MX.as<double>(), k, nm_.as<double>(), s));
    std::vector<double> hr(k), hm(k);
    NM_CUDA(cudaMemcpyAsync(hr.data(), nr.p, k * sizeof(double), cudaMemcpyDeviceToHost, s));
    NM_CUDA(cudaMemcpyAsync(hm.data(), nm_.p, k * sizeof(double), cudaMemcpyDeviceToHost, s));
    NM_CUDA(cudaStreamSynchronize(s));
    const double floor = 1e-3 * std::max(std::fabs(lam_lo), std::fabs(lam_hi));
    for (int i = 0; i < k; ++i)
        out.res[i] = std::sqrt(hr[i]) / (std::sqrt(hm[i]) * std::max(std::fabs(out.lam[i]), floor));
    if (X) {
        NM_TRY(X->alloc((size_t)n * k * sizeof(double)));
        NM_TRY(proj(V, ldv, X->as<double>()));
        NM_CUDA(cudaStreamSynchronize(s));
    }
    return NM_OK;
}

// ------------------------------------------------------------------ bounds
int spectrum_bounds(nm_problem* P, int steps, int k_M, uint64_t seed, double* lam_lo, double* lam_hi) {
    nm_ctx* ctx = P->ctx;
    cudaStream_t s = ctx->stream;
    const int64_t n = P->info.n;
    if (steps < 2) steps = 40;
    if (k_M < 2) k_M = 57;
    const int ldv = steps + 1;
    DevBuf V, W, MW, C, G, tmp;
    NM_TRY(V.alloc((size_t)n * ldv * sizeof(double)));
    NM_TRY(W.alloc((size_t)n * sizeof(double)));
    NM_TRY(MW.alloc((size_t)n * sizeof(double)));
    NM_TRY(C.alloc((size_t)ldv * sizeof(double)));
    NM_TRY(G.alloc(sizeof(double)));
    NM_TRY(tmp.alloc((size_t)n * sizeof(double)));
    NM_TRY(launch_philox_normal(n, seed, tmp.as<double>(), s));
    NM_TRY(launch_scale_copy<double>(n, 1, 1.0, tmp.as<double>(), 1, V.as<double>(), ldv, s));
    int ok = 1;
    NM_TRY(m_orth(P, V.as<double>(), ldv, 1, MW.as<double>(), G.as<double>(), &ok, s));
    if (!ok) return fail(NM_ENOTCONV, "start vector has zero M-norm");
    std::vector<double> T((size_t)steps * steps, 0.0);
    double beta_last = 0.0;
    int done = 0;
    Scratch<double> S;
    NM_TRY(get_scratch<double>(P, 1, S));
    for (int j = 0; j < steps; ++j) {
        const double* vj = V.as<double>() + j;
        // w = P_M K v_j
        NM_TRY(apply_K_t<double>(P, vj, ldv, S.W, 1, 1, k_M, S, S.XA, 1.0 / (0.5 * (kMassLo + kMassHi)), s));
        NM_TRY(mass_steps<double>(mats<double>(P), 1, k_M, kMassLo, kMassHi, S, nullptr, nullptr, nullptr,
                                  nullptr, nullptr, 0, W.as<double>(), 1, s));
        std::vector<double> hsum(j + 1, 0.0), hc(j + 1);
        for (int pass = 0; pass < 2; ++pass) {
            NM_TRY(apply_M_pub<double>(P, W.as<double>(), 1, MW.as<double>(), 1, 1, KRON_PLAIN, nullptr, s));
            NM_TRY(gemm_VtW(ctx, n, j + 1, 1, V.as<double>(), ldv, MW.as<double>(), 1, C.as<double>(), 0.0));
            NM_TRY(gemm_WmVC(ctx, n, j + 1, 1, -1.0, V.as<double>(), ldv, C.as<double>(), j + 1, W.as<double>(), 1));
            NM_CUDA(cudaMemcpyAsync(hc.data(), C.p, (j + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
            NM_CUDA(cudaStreamSynchronize(s));
            for (int i = 0; i <= j; ++i) hsum[i] += hc[i];
        }
        for (int i = 0; i <= j; ++i) T[(size_t)i + (size_t)j * steps] = hsum[i];
        NM_TRY(launch_scale_copy<double>(n, 1, 1.0, W.as<double>(), 1, V.as<double>() + j + 1, ldv, s));
        NM_TRY(m_orth(P, V.as<double>() + j + 1, ldv, 1, MW.as<double>(), G.as<double>(), &ok, s));
        double g = 0;
        NM_CUDA(cudaMemcpyAsync(&g, G.p, sizeof(double), cudaMemcpyDeviceToHost, s));
        NM_CUDA(cudaStreamSynchronize(s));
        beta_last = ok ? g : 0.0;
        done = j + 1;
        if (!ok) break;
    }
    // eigenvalues of the symmetrised projected matrix (host-tiny, done on device)
    const int m = done;
    std::vector<double> Tm((size_t)m * m);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) {
            const double a = i <= j ? T[(size_t)i + (size_t)j * steps] : T[(size_t)j + (size_t)i * steps];
            Tm[(size_t)i + (size_t)j * m] = a;
        }
    DevBuf Td, wd;
    NM_TRY(Td.alloc((size_t)m * m * sizeof(double)));
    NM_TRY(wd.alloc((size_t)m * sizeof(double)));
    NM_CUDA(cudaMemcpy(Td.p, Tm.data(), Tm.size() * sizeof(double), cudaMemcpyHostToDevice));
    NM_TRY(dense_eig(ctx, m, Td.as<double>(), nullptr, wd.as<double>()));
    std::vector<double> th(m), Sv((size_t)m * m);
    NM_CUDA(cudaMemcpy(th.data(), wd.p, m * sizeof(double), cudaMemcpyDeviceToHost));
    NM_CUDA(cudaMemcpy(Sv.data(), Td.p, Sv.size() * sizeof(double), cudaMemcpyDeviceToHost));
    const double r_hi = std::fabs(beta_last * Sv[(size_t)(m - 1) + (size_t)(m - 1) * m]);
    const double r_lo = std::fabs(beta_last * Sv[(size_t)(m - 1)]);
    // Upper end: Ritz value plus its residual bound, 1% margin. Lower end:
    // the smallest Ritz value (an upper bound of lambda_min) moved down by
    // 1e-6 lam_hi. The residual of the bottom Ritz value is not used: at the
    // clustered low end it is large and would push lam_lo far below the
    // spectrum, costing filter resolution exactly where slices sit; an
    // undershoot of delta only lets T_d grow to cosh(d sqrt(2 delta / e)),
    // about 1 for delta << e / d^2.
    // With self-gravitation the operator has a negative part of unknown
    // extent (the -C^T S C term lowers the rigid and the fluid modes), so
    // there the bottom Ritz value is moved down by its residual bound.
    const double hi = (th[m - 1] + r_hi) * 1.01;
    const double lo = P->sg.on ? std::min(0.0, th[0] - r_lo) - 1e-6 * hi : std::min(0.0, th[0]) - 1e-6 * hi;
    *lam_lo = lo;
    *lam_hi = hi;
    P->bounds_lo = lo;
    P->bounds_hi = hi;
    P->have_bounds = 1;
    P->bounds_key_steps = steps;
    P->bounds_key_kM = k_M;
    P->bounds_key_seed = seed;
    return NM_OK;
}

// ------------------------------------------------------------------ Lanczos
// One slice's filtered block Lanczos state (basis, projected matrix, filter).
struct SliceState {
    double lam_lo = 0, lam_hi = 0, tau = 0;
    std::vector<double> gamma;
    DevBuf V, MW, C, H, G;
    std::vector<double> Tfull;
    int j = 0;                    // block steps this slice has taken
    int blocks = 0, m_used = 0;
    bool active = true, converged = false, ok = true, taken = false;
    int nwanted = 0, nconv = 0;   // at the last block step
    int empty_checks = 0;         // consecutive converged checks that found no pair in the slice
    RRResult rr;
    nm_result* R = nullptr;
};

}  // namespace nm

// A filtered block Lanczos run of several slices in lockstep, advanced one
// block step at a time. The slices share the spectrum bounds, hence the
// Chebyshev map (c, e) and the recurrence; their current blocks are
// filtered together as one block with a per-slice gamma in the
// accumulation. Each slice has its own M-orthonormal basis, two-pass CGS,
// Cholesky-QR, projected matrix, convergence test and Rayleigh-Ritz, its
// own block counter, and leaves the batch when done; slices may join a
// running batch (nm_lanczos_add) and leave it (nm_lanczos_take).
struct nm_lanczos {
    nm_problem* P = nullptr;
    nm_slice_opts o{};
    int b = 0, d = 0, k_M = 0, k_P = 0, check = 1, mmax = 0, ldv = 0;
    double tol = 1e-6, conv_T = 1e-8, blo = 0, bhi = 0, c = 0, e = 0;
    std::deque<nm::SliceState> st;   // slices never move once added
    nm::DevBuf Ycat, Wcat, gtab, fin, fout;
    int cols_cap = 0, gtab_cap = 0;  // columns and slices the concatenated buffers hold
    double t_filter = 0.0;
    int j = 0;   // block steps taken by the run
    std::chrono::steady_clock::time_point t_start;
};

namespace nm {

// Filter, start block and first Cholesky-QR of a slice joining run L.
static int slice_init(nm_lanczos* L, SliceState& z, double lam_lo, double lam_hi, const double* start,
                      uint64_t seed) {
    nm_problem* P = L->P;
    cudaStream_t s = P->ctx->stream;
    const int64_t n = P->info.n;
    const int b = L->b, d = L->d, ldv = L->ldv;
    // lambda_lo = 0 takes the zero modes in; a negative edge stays as given
    z.lam_lo = lam_lo == 0 ? -1e-8 * L->bhi : lam_lo;
    z.lam_hi = lam_hi;
    z.gamma.resize(d + 1);
    jackson_step_coeffs(L->blo, L->bhi, z.lam_lo, z.lam_hi, d, z.gamma.data(), &L->c, &L->e);
    const double pa = cheb_sum(z.gamma, (z.lam_lo - L->c) / L->e), pb = cheb_sum(z.gamma, (z.lam_hi - L->c) / L->e);
    z.tau = z.lam_lo > L->blo ? 0.8 * std::min(pa, pb) : 0.8 * pb;
    NM_TRY(z.V.alloc((size_t)n * ldv * sizeof(double)));
    NM_TRY(z.MW.alloc((size_t)n * b * sizeof(double)));
    NM_TRY(z.C.alloc((size_t)ldv * b * sizeof(double)));
    NM_TRY(z.H.alloc((size_t)ldv * b * sizeof(double)));
    NM_TRY(z.G.alloc((size_t)b * b * sizeof(double)));
    z.Tfull.assign((size_t)L->mmax * L->mmax, 0.0);
    if (start) {
        NM_TRY(launch_scale_copy<double>(n, b, 1.0, start, b, z.V.as<double>(), ldv, s));
    } else {
        NM_TRY(launch_philox_normal(n * b, seed, z.MW.as<double>(), s));
        NM_TRY(launch_scale_copy<double>(n, b, 1.0, z.MW.as<double>(), b, z.V.as<double>(), ldv, s));
    }
    int ok = 1;
    NM_TRY(m_orth(P, z.V.as<double>(), ldv, b, z.MW.as<double>(), z.G.as<double>(), &ok, s));
    if (!ok) return fail(NM_ENOTCONV, "start block is rank deficient in the M inner product");
    return NM_OK;
}

// Room in the concatenated buffers for `slices` slices of b columns.
static int ensure_cat(nm_lanczos* L, int slices) {
    const int64_t n = L->P->info.n;
    if (slices * L->b > L->cols_cap) {
        const int cols = slices * L->b;
        L->Ycat.release();
        L->Wcat.release();
        NM_TRY(L->Ycat.alloc((size_t)n * cols * sizeof(double)));
        NM_TRY(L->Wcat.alloc((size_t)n * cols * sizeof(double)));
        L->cols_cap = cols;
    }
    if (slices > L->gtab_cap) {
        L->gtab.release();
        NM_TRY(L->gtab.alloc((size_t)(L->d + 1) * slices * sizeof(double)));
        L->gtab_cap = slices;
    }
    return NM_OK;
}

int lanczos_begin(nm_problem* P, const nm_slice_opts* o, int S, const double* lam_lo_in, const double* lam_hi_in,
                  nm_lanczos** out) {
    *out = nullptr;
    const int b = o->block;
    if (S < 1) return fail(NM_EINVAL, "need at least one slice");
    if (b < 1 || b > 64) return fail(NM_EINVAL, "block width must be in 1..64");
    if (o->degree < 1) return fail(NM_EINVAL, "degree must be >= 1");
    if (o->max_blocks < 2) return fail(NM_EINVAL, "max_blocks must be >= 2");
    for (int q = 0; q < S; ++q)
        if (!(lam_hi_in[q] > lam_lo_in[q])) return fail(NM_EINVAL, "slice needs lo < hi");
    std::unique_ptr<nm_lanczos> L(new (std::nothrow) nm_lanczos());
    if (!L) return fail(NM_ENOMEM, "host allocation failed");
    L->t_start = std::chrono::steady_clock::now();
    cudaStream_t s = P->ctx->stream;
    L->P = P;
    L->o = *o;
    L->o.start = nullptr;
    L->b = b;
    L->d = o->degree;
    L->k_M = o->k_M > 0 ? o->k_M : 57;
    L->k_P = o->k_P > 0 ? o->k_P : 57;
    L->tol = o->tol > 0 ? o->tol : 1e-6;
    L->check = o->check_every > 0 ? o->check_every : 1;
    L->conv_T = o->filter_prec == NM_F32 ? 1e-5 : 1e-8;
    L->mmax = b * o->max_blocks;
    L->ldv = L->mmax + b;
    const int bsteps = o->bounds_steps > 0 ? o->bounds_steps : 40;
    const uint64_t bseed = o->seed + 1;
    // The bounds depend only on (steps, k_M, seed): a problem keeps the last
    // estimate and reuses it for the same triple (options reset it).
    if (P->have_bounds && P->bounds_key_steps == bsteps && P->bounds_key_kM == L->k_M &&
        P->bounds_key_seed == bseed) {
        L->blo = P->bounds_lo;
        L->bhi = P->bounds_hi;
    } else {
        NM_TRY(spectrum_bounds(P, bsteps, L->k_M, bseed, &L->blo, &L->bhi));
    }
    // A slice that starts below the estimated bottom of the spectrum widens
    // the Chebyshev map down to its own edge: the caller expects
    // eigenvalues there, and outside the map the filter is unbounded.
    for (int q = 0; q < S; ++q)
        if (lam_lo_in[q] < 0 && lam_lo_in[q] < L->blo) L->blo = lam_lo_in[q] - 1e-6 * (L->bhi - lam_lo_in[q]);
    L->st.resize(S);
    for (int q = 0; q < S; ++q)
        NM_TRY(slice_init(L.get(), L->st[q], lam_lo_in[q], lam_hi_in[q], o->start,
                          o->seed + 0x9E3779B97F4A7C15ull * q));
    NM_TRY(ensure_cat(L.get(), S));
    NM_CUDA(cudaStreamSynchronize(s));
    *out = L.release();
    return NM_OK;
}

static bool slice_running(const nm_lanczos* L, const SliceState& z) {
    return z.active && !z.taken && z.j < L->o.max_blocks;
}

int lanczos_active(const nm_lanczos* L) {
    int a = 0;
    for (const SliceState& z : L->st) a += slice_running(L, z) ? 1 : 0;
    return a;
}

// One block step of every active slice: filter the current blocks, CGS2
// and Cholesky-QR of each slice's new block, its projected matrix, and,
// every check_every blocks of the slice (or at max_blocks), the convergence
// test and the Rayleigh-Ritz of the slices whose wanted Ritz values have
// converged.
int lanczos_step(nm_lanczos* L, int* active_out) {
    nm_problem* P = L->P;
    nm_ctx* ctx = P->ctx;
    cudaStream_t s = ctx->stream;
    const nm_slice_opts* o = &L->o;
    const int64_t n = P->info.n;
    const int b = L->b, d = L->d, ldv = L->ldv, mmax = L->mmax;
    std::vector<int> act;
    for (int q = 0; q < (int)L->st.size(); ++q)
        if (slice_running(L, L->st[q])) act.push_back(q);
    if (act.empty()) {
        *active_out = 0;
        return NM_OK;
    }
    // the active slices' blocks are filtered together, at most 64 columns
    // (one recurrence over the concatenated block) at a time
    const int per = std::max(1, 64 / b);
    NM_TRY(ensure_cat(L, std::min((int)act.size(), per)));
    for (size_t g0 = 0; g0 < act.size(); g0 += per) {
        const int Sa = (int)std::min<size_t>(per, act.size() - g0);
        const int B = Sa * b;
        // gamma table of the group's slices and their concatenated current blocks
        std::vector<double> gt((size_t)(d + 1) * Sa);
        for (int g = 0; g < Sa; ++g) {
            const SliceState& z = L->st[act[g0 + g]];
            for (int k = 0; k <= d; ++k) gt[(size_t)k * Sa + g] = z.gamma[k];
            NM_TRY(launch_scale_copy<double>(n, b, 1.0, z.V.as<double>() + (int64_t)z.j * b, ldv,
                                             L->Ycat.as<double>() + g * b, B, s));
        }
        NM_CUDA(cudaMemcpyAsync(L->gtab.p, gt.data(), gt.size() * sizeof(double), cudaMemcpyHostToDevice, s));
        NM_CUDA(cudaStreamSynchronize(s));
        auto t0 = std::chrono::steady_clock::now();
        GammaTable table{L->gtab.as<double>(), gt.data(), Sa, b};
        NM_TRY(filter_block(P, o->filter_prec, d, L->c, L->e, L->k_M, L->k_P, L->Ycat.as<double>(), B,
                            L->Wcat.as<double>(), B, &table, L->fin, L->fout, s));
        NM_CUDA(cudaStreamSynchronize(s));
        L->t_filter += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (P->Mr.tma_state == 1) NM_TRY(tma_status(P->Mr.tma.err, s));
        for (int g = 0; g < Sa; ++g) {
            SliceState& z = L->st[act[g0 + g]];
            const int j = z.j;
            const int m = (j + 1) * b;
            double* W = L->Wcat.as<double>() + g * b;   // ld B
            // CGS2 against the slice's basis in the M inner product
            NM_CUDA(cudaMemsetAsync(z.H.p, 0, (size_t)m * b * sizeof(double), s));
            for (int pass = 0; pass < 2; ++pass) {
                NM_TRY(apply_M_pub<double>(P, W, B, z.MW.as<double>(), b, b, KRON_PLAIN, nullptr, s));
                NM_TRY(gemm_VtW(ctx, n, m, b, z.V.as<double>(), ldv, z.MW.as<double>(), b, z.C.as<double>(), 0.0));
                NM_TRY(gemm_WmVC(ctx, n, m, b, -1.0, z.V.as<double>(), ldv, z.C.as<double>(), m, W, B));
                const double one = 1.0;
                NM_CUBLAS(cublasDaxpy(ctx->cublas, m * b, &one, z.C.as<double>(), 1, z.H.as<double>(), 1));
            }
            std::vector<double> hH((size_t)m * b);
            NM_CUDA(cudaMemcpyAsync(hH.data(), z.H.p, hH.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
            double* Vn = z.V.as<double>() + (int64_t)(j + 1) * b;
            NM_TRY(launch_scale_copy<double>(n, b, 1.0, W, B, Vn, ldv, s));
            int ok = 1;
            NM_TRY(m_orth(P, Vn, ldv, b, z.MW.as<double>(), z.G.as<double>(), &ok, s));
            z.ok = ok != 0;
            std::vector<double> hR((size_t)b * b);
            NM_CUDA(cudaMemcpy(hR.data(), z.G.p, hR.size() * sizeof(double), cudaMemcpyDeviceToHost));
            for (int cc = 0; cc < b; ++cc)
                for (int r = 0; r < m; ++r)
                    z.Tfull[(size_t)r + (size_t)(j * b + cc) * mmax] = hH[(size_t)r + (size_t)cc * m];
            z.j = j + 1;
            z.blocks = j + 1;
            z.m_used = m;
            std::vector<double> Tm((size_t)m * m);
            for (int r = 0; r < m; ++r)
                for (int cc = 0; cc < m; ++cc)
                    Tm[(size_t)r + (size_t)cc * m] = r <= cc ? z.Tfull[(size_t)r + (size_t)cc * mmax]
                                                             : z.Tfull[(size_t)cc + (size_t)r * mmax];
            DevBuf Td, wd;
            NM_TRY(Td.alloc(Tm.size() * sizeof(double)));
            NM_TRY(wd.alloc(m * sizeof(double)));
            NM_CUDA(cudaMemcpy(Td.p, Tm.data(), Tm.size() * sizeof(double), cudaMemcpyHostToDevice));
            NM_TRY(dense_eig(ctx, m, Td.as<double>(), nullptr, wd.as<double>()));
            std::vector<double> th(m), Sv((size_t)m * m);
            NM_CUDA(cudaMemcpy(th.data(), wd.p, m * sizeof(double), cudaMemcpyDeviceToHost));
            NM_CUDA(cudaMemcpy(Sv.data(), Td.p, Sv.size() * sizeof(double), cudaMemcpyDeviceToHost));
            int nwanted = 0, nconv = 0;
            for (int i = 0; i < m; ++i) {
                if (th[i] < z.tau) continue;
                ++nwanted;
                double r2 = 0;
                if (ok)
                    for (int r = 0; r < b; ++r) {
                        double v = 0;
                        for (int qq = r; qq < b; ++qq)
                            v += hR[(size_t)r + (size_t)qq * b] * Sv[(size_t)(m - b + qq) + (size_t)i * m];
                        r2 += v * v;
                    }
                if (std::sqrt(r2) <= L->conv_T * std::max(std::fabs(th[i]), 1.0)) ++nconv;
            }
            z.nwanted = nwanted;
            z.nconv = nconv;
            if (o->log_every > 0 && (j + 1) % o->log_every == 0)
                fprintf(stderr, "[nm] slice %d block %d m=%d wanted=%d converged=%d filter %.1fs total %.1fs\n",
                        act[g0 + g],
                        j + 1, m, nwanted, nconv, L->t_filter,
                        std::chrono::duration<double>(std::chrono::steady_clock::now() - L->t_start).count());
            const bool last = j + 1 == o->max_blocks || !ok;
            if ((nwanted > 0 && nconv == nwanted && (j + 1) % L->check == 0) || last) {
                if (!z.R) {
                    z.R = new (std::nothrow) nm_result();
                    if (!z.R) return fail(NM_ENOMEM, "host allocation failed");
                }
                // With every wanted Ritz value of p(B) converged, the slice's
                // pairs are the pencil's Ritz pairs that lie in the span of
                // their Ritz vectors (the top nwanted eigenvectors of T)
                const bool conv_all = nwanted > 0 && nconv == nwanted;
                NM_TRY(rayleigh_ritz(P, z.V.as<double>(), ldv, m, z.lam_lo, z.lam_hi, &z.R->X, z.rr,
                                     conv_all ? Sv.data() + (size_t)(m - nwanted) * m : nullptr, nwanted));
                bool all = z.rr.k > 0;
                for (double r : z.rr.res) all = all && r <= L->tol;
                // An empty slice: every wanted Ritz value of p(B) has converged
                // (all of them belong to eigenvalues outside the slice) and no
                // pencil pair lies in the slice, at two consecutive checks
                // from the fourth block on. An eigenvalue inside the slice has
                // p >= tau, so it would be among the wanted ones.
                z.empty_checks = conv_all && z.rr.k == 0 ? z.empty_checks + 1 : 0;
                if (z.empty_checks >= 2 && j + 1 >= 4) all = true;
                if (all || last) {
                    z.converged = all;
                    z.active = false;
                }
            }
        }
    }
    L->j += 1;
    *active_out = lanczos_active(L);
    return NM_OK;
}

// Result of slice q (a Rayleigh-Ritz on its current basis if it has none
// yet); the slice leaves the run and its basis is released.
static int slice_result(nm_lanczos* L, SliceState& z, nm_result** out) {
    nm_problem* P = L->P;
    *out = nullptr;
    if (!z.R) {
        z.R = new (std::nothrow) nm_result();
        if (!z.R) return fail(NM_ENOMEM, "host allocation failed");
        if (z.m_used > 0) {
            NM_TRY(rayleigh_ritz(P, z.V.as<double>(), L->ldv, z.m_used, z.lam_lo, z.lam_hi, &z.R->X, z.rr));
        } else {
            // no block step taken: the start block is the basis
            NM_TRY(rayleigh_ritz(P, z.V.as<double>(), L->ldv, L->b, z.lam_lo, z.lam_hi, &z.R->X, z.rr));
            z.m_used = L->b;
        }
    }
    nm_result* R = z.R;
    R->lambda = z.rr.lam;
    R->resid = z.rr.res;
    R->info.k = z.rr.k;
    R->info.n = P->info.n;
    R->info.blocks = z.blocks;
    R->info.m = z.m_used;
    R->info.filter_applications = (int64_t)z.blocks * L->b;
    R->info.lam_lo = L->blo;
    R->info.lam_hi = L->bhi;
    R->info.seconds_filter = L->t_filter;
    R->info.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - L->t_start).count();
    z.R = nullptr;
    z.active = false;
    z.taken = true;
    for (DevBuf* buf : {&z.V, &z.MW, &z.C, &z.H, &z.G}) buf->release();
    std::vector<double>().swap(z.Tfull);
    *out = R;
    return NM_OK;
}

// Results of every slice not taken yet (out[q] = nullptr for taken ones).
// NM_ENOTCONV if a slice did not pass tol; the results are returned all the
// same. Ownership of the results moves to the caller.
int lanczos_finish(nm_lanczos* L, nm_result** out) {
    const int S = (int)L->st.size();
    for (int q = 0; q < S; ++q) out[q] = nullptr;
    int rc = NM_OK;
    for (int q = 0; q < S; ++q) {
        SliceState& z = L->st[q];
        if (z.taken) continue;
        const bool conv = z.converged;
        NM_TRY(slice_result(L, z, out + q));
        if (!conv) rc = NM_ENOTCONV;
    }
    if (rc != NM_OK) return fail(rc, "a slice did not converge within max_blocks");
    return NM_OK;
}

int lanczos_take(nm_lanczos* L, int q, nm_result** out) {
    *out = nullptr;
    if (q < 0 || q >= (int)L->st.size()) return fail(NM_EINVAL, "slice index out of range");
    SliceState& z = L->st[q];
    if (z.taken) return fail(NM_EINVAL, "slice already taken");
    const bool conv = z.converged;
    NM_TRY(slice_result(L, z, out));
    if (!conv) return fail(NM_ENOTCONV, "the slice did not converge (its current Ritz pairs are returned)");
    return NM_OK;
}

int lanczos_add(nm_lanczos* L, double lam_lo, double lam_hi, uint64_t seed, const double* start, int* index) {
    *index = -1;
    if (!(lam_hi > lam_lo)) return fail(NM_EINVAL, "slice needs lo < hi");
    L->st.emplace_back();
    const int q = (int)L->st.size() - 1;
    const int rc = slice_init(L, L->st[q], lam_lo, lam_hi, start, seed);
    if (rc != NM_OK) {
        SliceState& z = L->st[q];
        z.active = false;
        z.taken = true;
        for (DevBuf* buf : {&z.V, &z.MW, &z.C, &z.H, &z.G}) buf->release();
        return rc;
    }
    NM_CUDA(cudaStreamSynchronize(L->P->ctx->stream));
    *index = q;
    return NM_OK;
}

int lanczos_nslices(const nm_lanczos* L) { return (int)L->st.size(); }

int lanczos_state(const nm_lanczos* L, int slice, nm_lanczos_info* out) {
    if (slice < 0 || slice >= (int)L->st.size()) return fail(NM_EINVAL, "slice index out of range");
    const SliceState& z = L->st[slice];
    out->blocks = z.blocks;
    out->m = z.m_used;
    out->active = slice_running(L, z) ? 1 : 0;
    out->converged = z.converged ? 1 : 0;
    out->wanted = z.nwanted;
    out->ritz_converged = z.nconv;
    out->seconds_filter = L->t_filter;
    return NM_OK;
}

nm_ctx* lanczos_ctx(const nm_lanczos* L) { return L->P->ctx; }

void lanczos_free(nm_lanczos* L) {
    if (!L) return;
    for (SliceState& z : L->st) {
        delete z.R;
        z.R = nullptr;
    }
    delete L;
}

// Filtered block Lanczos for S slices in lockstep (S = 1: nm_lanczos_slice):
// begin, block steps until no slice is active, finish.
int lanczos_multi(nm_problem* P, const nm_slice_opts* o, int S, const double* lam_lo_in, const double* lam_hi_in,
                  nm_result** out) {
    for (int q = 0; q < S; ++q) out[q] = nullptr;
    nm_lanczos* L = nullptr;
    int rc = lanczos_begin(P, o, S, lam_lo_in, lam_hi_in, &L);
    if (rc != NM_OK) return rc;
    int active = 1;
    while (active > 0 && rc == NM_OK) rc = lanczos_step(L, &active);
    if (rc == NM_OK) rc = lanczos_finish(L, out);
    lanczos_free(L);
    return rc;
}

int lanczos_slice(nm_problem* P, const nm_slice_opts* o, nm_result** out) {
    if (!P->have_interval) return fail(NM_EINVAL, "call nm_set_interval first");
    return lanczos_multi(P, o, 1, &P->lo, &P->hi, out);
}

// ------------------------------------------------------------------ Ritz entry
__global__ void interleave_complex_kernel(int64_t count, const double* re, const double* im, double* out) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
         t += (int64_t)gridDim.x * blockDim.x) {
        out[2 * t] = re[t];
        out[2 * t + 1] = im[t];
    }
}

int ritz(nm_problem* P, nm_ritz_mode mode, const double* V, int64_t ldv, int m, const double* lam_e,
         nm_result** out) {
    auto t_start = std::chrono::steady_clock::now();
    nm_ctx* ctx = P->ctx;
    cudaStream_t s = ctx->stream;
    const int64_t n = P->info.n;
    if (m < 1 || !V || ldv < m) return fail(NM_EINVAL, "ritz needs m >= 1, V and ldv >= m");
    if (!P->have_interval) return fail(NM_EINVAL, "call nm_set_interval first");
    nm_result* R = new (std::nothrow) nm_result();
    if (!R) return fail(NM_ENOMEM, "host allocation failed");
    std::unique_ptr<nm_result> guard(R);
    if (mode == NM_RITZ_PENCIL) {
        const double lam_lo = P->lo == 0 ? -1e-8 * std::max(1.0, std::fabs(P->hi)) : P->lo;
        RRResult rr;
        NM_TRY(rayleigh_ritz(P, V, ldv, m, lam_lo, P->hi, &R->X, rr));
        R->lambda = rr.lam;
        R->resid = rr.res;
        R->info.k = rr.k;
        R->info.n = n;
        R->info.m = m;
    } else if (mode == NM_RITZ_ROTATING) {
        if (!lam_e) return fail(NM_EINVAL, "rotating mode needs the Ritz values lam_e");
        for (int i = 0; i < m; ++i)
            if (!(lam_e[i] > 0)) return fail(NM_EINVAL, "rotating mode needs lam_e > 0");
        // Q = X^T R X (real skew), R X = (M_rho (x) [Omega]_x) X
        DevBuf RX, Q;
        NM_TRY(RX.alloc((size_t)n * m * sizeof(double)));
        NM_TRY(Q.alloc((size_t)m * m * sizeof(double)));
        NM_TRY(apply_cols(P, 2, V, ldv, RX.as<double>(), m, m, 0, s));
        NM_TRY(gemm_VtW(ctx, n, m, m, V, ldv, RX.as<double>(), m, Q.as<double>(), 0.0));
        std::vector<double> hQ((size_t)m * m);
        NM_CUDA(cudaMemcpyAsync(hQ.data(), Q.p, hQ.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        NM_CUDA(cudaStreamSynchronize(s));
        // pencil [[0, L], [L, 2iQ]] y = w [[L, 0], [0, I]] y (eq. sublinear0), complex Hermitian
        const int m2 = 2 * m;
        std::vector<cuDoubleComplex> A((size_t)m2 * m2, make_cuDoubleComplex(0, 0)), B(A);
        for (int i = 0; i < m; ++i) {
            A[(size_t)i + (size_t)(m + i) * m2] = make_cuDoubleComplex(lam_e[i], 0);
            A[(size_t)(m + i) + (size_t)i * m2] = make_cuDoubleComplex(lam_e[i], 0);
            B[(size_t)i + (size_t)i * m2] = make_cuDoubleComplex(lam_e[i], 0);
            B[(size_t)(m + i) + (size_t)(m + i) * m2] = make_cuDoubleComplex(1, 0);
        }
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) {
                // Hermitian part of 2iQ: Q skew => 2iQ Hermitian; symmetrise against rounding
                const double q = 0.5 * (hQ[(size_t)i + (size_t)j * m] - hQ[(size_t)j + (size_t)i * m]);
                A[(size_t)(m + i) + (size_t)(m + j) * m2] = make_cuDoubleComplex(0, 2.0 * q);
            }
        DevBuf Ad, Bd, wd, info;
        NM_TRY(Ad.alloc(A.size() * sizeof(cuDoubleComplex)));
        NM_TRY(Bd.alloc(B.size() * sizeof(cuDoubleComplex)));
        NM_TRY(wd.alloc(m2 * sizeof(double)));
        NM_TRY(info.alloc(sizeof(int)));
        NM_CUDA(cudaMemcpy(Ad.p, A.data(), A.size() * sizeof(cuDoubleComplex), cudaMemcpyHostToDevice));
        NM_CUDA(cudaMemcpy(Bd.p, B.data(), B.size() * sizeof(cuDoubleComplex), cudaMemcpyHostToDevice));
        int lwork = 0;
        NM_CUSOLVER(cusolverDnZhegvd_bufferSize(ctx->cusolver, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR,
                                                CUBLAS_FILL_MODE_UPPER, m2, Ad.as<cuDoubleComplex>(), m2,
                                                Bd.as<cuDoubleComplex>(), m2, wd.as<double>(), &lwork));
        DevBuf work;
        NM_TRY(work.alloc(std::max(lwork, 1) * sizeof(cuDoubleComplex)));
        NM_CUSOLVER(cusolverDnZhegvd(ctx->cusolver, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR,
                                     CUBLAS_FILL_MODE_UPPER, m2, Ad.as<cuDoubleComplex>(), m2,
                                     Bd.as<cuDoubleComplex>(), m2, wd.as<double>(), work.as<cuDoubleComplex>(),
                                     lwork, info.as<int>()));
        int h = 0;
        NM_CUDA(cudaStreamSynchronize(s));
        NM_CUDA(cudaMemcpy(&h, info.p, sizeof(int), cudaMemcpyDeviceToHost));
        if (h != 0) return fail(NM_ENOTCONV, "rotating dense eigensolver failed");
        std::vector<double> w(m2);
        std::vector<cuDoubleComplex> Y((size_t)m2 * m2);
        NM_CUDA(cudaMemcpy(w.data(), wd.p, m2 * sizeof(double), cudaMemcpyDeviceToHost));
        NM_CUDA(cudaMemcpy(Y.data(), Ad.p, Y.size() * sizeof(cuDoubleComplex), cudaMemcpyDeviceToHost));
        const double wlo = P->lo > 0 ? std::sqrt(P->lo) : 0.0, whi = std::sqrt(std::max(P->hi, 0.0));
        std::vector<int> sel;
        for (int i = 0; i < m2; ++i)
            if (w[i] >= wlo && w[i] <= whi) sel.push_back(i);
        const int k = (int)sel.size();
        R->lambda.resize(k);
        R->resid.assign(k, 0.0);
        R->info.k = k;
        R->info.n = n;
        R->info.m = m;
        R->info.complex_vectors = 1;
        if (k > 0) {
            // y_top (m x k) real and imaginary parts, col-major; u = X_e y_top
            std::vector<double> yr((size_t)m * k), yi((size_t)m * k);
            for (int c = 0; c < k; ++c) {
                R->lambda[c] = w[sel[c]];
                for (int i = 0; i < m; ++i) {
                    yr[(size_t)i + (size_t)c * m] = cuCreal(Y[(size_t)i + (size_t)sel[c] * m2]);
                    yi[(size_t)i + (size_t)c * m] = cuCimag(Y[(size_t)i + (size_t)sel[c] * m2]);
                }
            }
            DevBuf yrd, yid, Ur, Ui;
            NM_TRY(yrd.alloc(yr.size() * sizeof(double)));
            NM_TRY(yid.alloc(yi.size() * sizeof(double)));
            NM_TRY(Ur.alloc((size_t)n * k * sizeof(double)));
            NM_TRY(Ui.alloc((size_t)n * k * sizeof(double)));
            NM_CUDA(cudaMemcpy(yrd.p, yr.data(), yr.size() * sizeof(double), cudaMemcpyHostToDevice));
            NM_CUDA(cudaMemcpy(yid.p, yi.data(), yi.size() * sizeof(double), cudaMemcpyHostToDevice));
            NM_TRY(gemm_VS(ctx, n, m, k, V, ldv, yrd.as<double>(), m, Ur.as<double>(), k));
            NM_TRY(gemm_VS(ctx, n, m, k, V, ldv, yid.as<double>(), m, Ui.as<double>(), k));
            // full quadratic residual ||w^2 M u - 2 i w R u - K u|| / ||w^2 M u|| (reported, not gated)
            DevBuf KUr, KUi, MUr, MUi, RUr, RUi;
            for (DevBuf* d : {&KUr, &KUi, &MUr, &MUi, &RUr, &RUi}) NM_TRY(d->alloc((size_t)n * k * sizeof(double)));
            NM_TRY(apply_cols(P, 0, Ur.as<double>(), k, KUr.as<double>(), k, k, 80, s));
            NM_TRY(apply_cols(P, 0, Ui.as<double>(), k, KUi.as<double>(), k, k, 80, s));
            NM_TRY(apply_cols(P, 1, Ur.as<double>(), k, MUr.as<double>(), k, k, 0, s));
            NM_TRY(apply_cols(P, 1, Ui.as<double>(), k, MUi.as<double>(), k, k, 0, s));
            NM_TRY(apply_cols(P, 2, Ur.as<double>(), k, RUr.as<double>(), k, k, 0, s));
            NM_TRY(apply_cols(P, 2, Ui.as<double>(), k, RUi.as<double>(), k, k, 0, s));
            NM_CUDA(cudaStreamSynchronize(s));
            std::vector<double> hK[2], hM[2], hRr[2];
            for (int p = 0; p < 2; ++p) {
                hK[p].resize((size_t)n * k);
                hM[p].resize((size_t)n * k);
                hRr[p].resize((size_t)n * k);
            }
            NM_CUDA(cudaMemcpy(hK[0].data(), KUr.p, (size_t)n * k * 8, cudaMemcpyDeviceToHost));
            NM_CUDA(cudaMemcpy(hK[1].data(), KUi.p, (size_t)n * k * 8, cudaMemcpyDeviceToHost));
            NM_CUDA(cudaMemcpy(hM[0].data(), MUr.p, (size_t)n * k * 8, cudaMemcpyDeviceToHost));
            NM_CUDA(cudaMemcpy(hM[1].data(), MUi.p, (size_t)n * k * 8, cudaMemcpyDeviceToHost));
            NM_CUDA(cudaMemcpy(hRr[0].data(), RUr.p, (size_t)n * k * 8, cudaMemcpyDeviceToHost));
            NM_CUDA(cudaMemcpy(hRr[1].data(), RUi.p, (size_t)n * k * 8, cudaMemcpyDeviceToHost));
            for (int c = 0; c < k; ++c) {
                const double om = R->lambda[c];
                double num = 0, den = 0;
                for (int64_t i = 0; i < n; ++i) {
                    const size_t q = (size_t)i * k + c;
                    // w^2 M u - 2 i w R u - K u
                    const double re = om * om * hM[0][q] + 2 * om * hRr[1][q] - hK[0][q];
                    const double im = om * om * hM[1][q] - 2 * om * hRr[0][q] - hK[1][q];
                    num += re * re + im * im;
                    den += om * om * om * om * (hM[0][q] * hM[0][q] + hM[1][q] * hM[1][q]);
                }
                R->resid[c] = den > 0 ? std::sqrt(num / den) : 0.0;
            }
            NM_TRY(R->X.alloc((size_t)n * k * 2 * sizeof(double)));
            interleave_complex_kernel<<<(unsigned)std::min<int64_t>((n * k + 255) / 256, 4864), 256, 0, s>>>(
                n * k, Ur.as<double>(), Ui.as<double>(), R->X.as<double>());
            count_launch();
        NM_CUDA(cudaGetLastError());
            NM_CUDA(cudaStreamSynchronize(s));
        }
    } else {
        return fail(NM_EINVAL, "unknown ritz mode");
    }
    R->info.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    *out = guard.release();
    return NM_OK;
}

}  // namespace nm
