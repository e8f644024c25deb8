// FP64-accurate dense products on the tensor cores by operand splitting.
//
// The dense algebra of the filtered block Lanczos (Sec. 6.2) is two product
// shapes over the basis V (n rows, n ~ 1e6):
//   TN:  C (I x J) = alpha X^T Y + beta C,  X: n x I, Y: n x J  (the block
//        Gram-Schmidt coefficients V^T M W, the Ritz projections V^T K V,
//        V^T M V and the Coriolis projection X^T R X, Sec. 7);
//   NN:  D (n x J) = alpha X Y + beta D,    X: n x I, Y: I x J  (W -= V C,
//        the Ritz vectors X = V S).
// GB300's FP64 units run at 1/64 of its float units and its tensor cores
// take no FP64 here, so both run as bf16 tensor-core products of exact
// operand slices (the error-free splitting of Ozaki, Ogita, Oishi and Rump,
// 2012):
//  - within a contraction chunk of 64 terms, every row i of X and column j
//    of Y gets the exponent E_i (F_j) of its largest entry; an entry's 53-bit
//    mantissa, shifted right by E_i minus its own exponent, is cut from the
//    top into eight 7-bit pieces t_1..t_8 (the last holds the 4 lowest bits,
//    shifted up by 3), so x = sign 2^(E_i - 1029) sum_p t_p 2^(-7(p-1))
//    exactly up to the bits below 2^-53 of the row's largest entry;
//  - every piece is an integer in [-127, 127], exact in bf16; a product of
//    two is below 2^14 and the sum over the chunk of the (at most 8) piece
//    pairs of one diagonal d = p + q - 2 is below 8 * 64 * 127^2 < 2^24, so
//    the float accumulation of the tensor cores (mma.sync m16n8k16, bf16
//    in, f32 out) is exact;
//  - the chunk's contribution sum_{d=0..7} 2^(-7d) acc_d 2^(E_i + F_j - 2058)
//    is added in FP64; the diagonals d >= 8 (weight <= 2^-56 of the product
//    of the two largest entries) are dropped.
// The result thus carries FP64-level error (relative to the products of
// each row's and column's largest entries) at 36 bf16 products per term.
// TN splits the long contraction over CTAs into a fixed number of parts
// summed in order by a second kernel, so every result is deterministic.
#include <algorithm>
#include <cstdint>

#include "kernels.h"
#include "nm_internal.h"

namespace nm {

namespace {

constexpr int kWarps = 4;
constexpr int kThreads = 32 * kWarps;
constexpr int kTileI = 16 * kWarps;    // output rows per CTA (16 per warp)
constexpr int kTileJ = 16;             // output columns per CTA (two n8 tiles)
constexpr int kChunk = 64;             // contraction terms per exact accumulation
constexpr int kSlices = 8;             // 7-bit pieces per operand
constexpr int kDiag = 8;               // kept diagonals d = p + q - 2 = 0..7
constexpr int kLdX = kChunk + 2;       // smem row stride of the X tile (doubles)
constexpr int kLdY = kChunk + 2;       // smem row stride of the Y tile (stored j-major)

// Biased exponent used for alignment (subnormals and zero count as 1).
__device__ __forceinline__ int exp_of(double v) {
    const int e = (int)((__double_as_longlong(v) >> 52) & 0x7FF);
    return e == 0 ? 1 : e;
}

// Eight 7-bit pieces of v aligned to exponent E (E >= exponent of v), as
// signed floats (integers in [-127, 127]).
__device__ __forceinline__ void slices(double v, int E, float* t) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((bits >> 52) & 0x7FF);
    unsigned long long m = bits & 0xFFFFFFFFFFFFFull;
    if (e != 0) m |= 1ull << 52;
    const int shift = E - (e == 0 ? 1 : e);
    m = shift >= 64 ? 0ull : (m >> shift);
    const float sg = (bits >> 63) ? -1.f : 1.f;
#pragma unroll
    for (int p = 0; p < 7; ++p) t[p] = sg * (float)(unsigned)((m >> (46 - 7 * p)) & 0x7Full);
    t[7] = sg * (float)(unsigned)((m << 3) & 0x7Full);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

struct Shape {
    // X(i, k) = xt ? X[k * ldx + i] : X[i * ldx + k]
    // Y(k, j) = ycm ? Y[k + j * ldy] : Y[k * ldy + j]
    const double* X;
    int64_t ldx;
    const double* Y;
    int64_t ldy;
    int64_t I, J, K;       // output rows, columns, contraction length
    int64_t k_per_part;    // contraction terms per split part (multiple of kChunk)
    // output: part p of TN writes P[p][i + j * I]; NN writes D
    double* P;
    double* D;
    int64_t ldd;
    double alpha, beta;
};

// One CTA: output tile rows i0 .. i0 + 63, columns j0 .. j0 + 15, contraction
// terms [k_begin, k_end) in chunks of 64.
template <bool XT, bool YCM, bool NN>
__global__ void __launch_bounds__(kThreads) ozaki_kernel(const Shape sh) {
    __shared__ double Xs[kTileI * kLdX];       // Xs[i][k]
    __shared__ double Ys[kTileJ * kLdY];       // Ys[j][k]
    __shared__ int Ex[kTileI], Fy[kTileJ];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gid = lane >> 2, tig = lane & 3;
    const int64_t i0 = (int64_t)blockIdx.x * kTileI;
    const int64_t j0 = (int64_t)blockIdx.y * kTileJ;
    const int part = blockIdx.z;
    const int64_t k_begin = (int64_t)part * sh.k_per_part;
    const int64_t k_end = sh.K < k_begin + sh.k_per_part ? sh.K : k_begin + sh.k_per_part;
    double out[2][4];
#pragma unroll
    for (int n = 0; n < 2; ++n)
#pragma unroll
        for (int r = 0; r < 4; ++r) out[n][r] = 0.0;
    for (int64_t k0 = k_begin; k0 < k_end; k0 += kChunk) {
        const int kc = (int)(k_end - k0 < kChunk ? k_end - k0 : kChunk);
        if (tid < kTileI) Ex[tid] = 1;
        if (tid < kTileJ) Fy[tid] = 1;
        __syncthreads();
        // stage X (64 x kc) and Y (kc x 16) in FP64, zero-padded, with the
        // row / column maxima of the exponents
        if (XT) {
            // X[k][i]: i contiguous; thread -> (i = tid & 63, k = (tid >> 6) + 2 s)
            const int ii = tid & 63;
            int emax = 1;
            for (int kk = tid >> 6; kk < kChunk; kk += kThreads / 64) {
                double v = 0.0;
                if (kk < kc && i0 + ii < sh.I) v = __ldg(sh.X + (k0 + kk) * sh.ldx + i0 + ii);
                Xs[ii * kLdX + kk] = v;
                emax = max(emax, exp_of(v));
            }
            atomicMax(&Ex[ii], emax);
        } else {
            // X[i][k]: k contiguous; warp w -> rows w, w + 4, ...; lane -> k
            for (int ii = warp; ii < kTileI; ii += kWarps) {
                int emax = 1;
                for (int kk = lane; kk < kChunk; kk += 32) {
                    double v = 0.0;
                    if (kk < kc && i0 + ii < sh.I) v = __ldg(sh.X + (i0 + ii) * sh.ldx + k0 + kk);
                    Xs[ii * kLdX + kk] = v;
                    emax = max(emax, exp_of(v));
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
                if (lane == 0) Ex[ii] = emax;
            }
        }
        if (YCM) {
            // Y[k + j ldy]: k contiguous; warp w -> columns w, w + 4, ...
            for (int jj = warp; jj < kTileJ; jj += kWarps) {
                int emax = 1;
                for (int kk = lane; kk < kChunk; kk += 32) {
                    double v = 0.0;
                    if (kk < kc && j0 + jj < sh.J) v = __ldg(sh.Y + (k0 + kk) + (j0 + jj) * sh.ldy);
                    Ys[jj * kLdY + kk] = v;
                    emax = max(emax, exp_of(v));
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
                if (lane == 0) Fy[jj] = emax;
            }
        } else {
            // Y[k ldy + j]: j contiguous; thread -> (j = tid & 15, k = (tid >> 4) + 8 s)
            const int jj = tid & 15;
            int emax = 1;
            for (int kk = tid >> 4; kk < kChunk; kk += kThreads / 16) {
                double v = 0.0;
                if (kk < kc && j0 + jj < sh.J) v = __ldg(sh.Y + (k0 + kk) * sh.ldy + j0 + jj);
                Ys[jj * kLdY + kk] = v;
                emax = max(emax, exp_of(v));
            }
            atomicMax(&Fy[jj], emax);
        }
        __syncthreads();
        // warp: rows i0 + 16 warp + (gid, gid + 8); columns j0 + 8 n + (2 tig, 2 tig + 1)
        const int ra = 16 * warp + gid, rb = ra + 8;
        const int Ea = Ex[ra], Eb = Ex[rb];
        float acc[kDiag][2][4];
#pragma unroll
        for (int d = 0; d < kDiag; ++d)
#pragma unroll
            for (int n = 0; n < 2; ++n)
#pragma unroll
                for (int r = 0; r < 4; ++r) acc[d][n][r] = 0.f;
        for (int ks = 0; ks < kChunk; ks += 16) {
            // A fragments of the eight slices: rows (ra, rb), k = ks + 2 tig + {0, 1} (+ 8)
            uint32_t a[kSlices][4];
            {
                float t0[kSlices], t1[kSlices];
                const int kk = ks + 2 * tig;
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int row = (h & 1) ? rb : ra;
                    const int E = (h & 1) ? Eb : Ea;
                    const int kq = kk + ((h & 2) ? 8 : 0);
                    slices(Xs[row * kLdX + kq], E, t0);
                    slices(Xs[row * kLdX + kq + 1], E, t1);
#pragma unroll
                    for (int p = 0; p < kSlices; ++p) a[p][h] = pack_bf16(t0[p], t1[p]);
                }
            }
#pragma unroll
            for (int n = 0; n < 2; ++n) {
                // B fragments: column 8 n + gid, k = ks + 2 tig + {0, 1} (+ 8)
                uint32_t b[kSlices][2];
                const int col = 8 * n + gid;
                const int F = Fy[col];
                float t0[kSlices], t1[kSlices];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int kq = ks + 2 * tig + 8 * h;
                    slices(Ys[col * kLdY + kq], F, t0);
                    slices(Ys[col * kLdY + kq + 1], F, t1);
#pragma unroll
                    for (int p = 0; p < kSlices; ++p) b[p][h] = pack_bf16(t0[p], t1[p]);
                }
#pragma unroll
                for (int p = 0; p < kSlices; ++p)
#pragma unroll
                    for (int q = 0; q < kSlices; ++q)
                        if (p + q < kDiag) mma_bf16(acc[p + q][n], a[p], b[q]);
            }
        }
        // exact chunk sums -> FP64
#pragma unroll
        for (int n = 0; n < 2; ++n) {
            const int c0 = 8 * n + 2 * tig;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                double s = 0.0;
#pragma unroll
                for (int d = kDiag - 1; d >= 0; --d) s = s * (1.0 / 128.0) + (double)acc[d][n][r];
                const int E = (r < 2) ? Ea : Eb;
                const int F = Fy[c0 + (r & 1)];
                out[n][r] += ldexp(s, E + F - 2058);
            }
        }
        __syncthreads();   // the tiles are restaged for the next chunk
    }
    // write: TN -> its part of the workspace, NN -> D (alpha, beta applied)
#pragma unroll
    for (int n = 0; n < 2; ++n)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int64_t i = i0 + 16 * warp + gid + ((r >= 2) ? 8 : 0);
            const int64_t j = j0 + 8 * n + 2 * tig + (r & 1);
            if (i >= sh.I || j >= sh.J) continue;
            if (NN) {
                double* d = sh.D + i * sh.ldd + j;
                *d = sh.alpha * out[n][r] + (sh.beta == 0.0 ? 0.0 : sh.beta * *d);
            } else {
                sh.P[(int64_t)part * sh.I * sh.J + i + j * sh.I] = out[n][r];
            }
        }
}

// C[i + j ldc] = alpha sum_p P[p][i + j I] + beta C (parts summed in order).
__global__ void ozaki_reduce_kernel(int64_t I, int64_t J, int parts, const double* P, double alpha, double beta,
                                    double* C, int64_t ldc) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < I * J; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t % I, j = t / I;
        double s = 0.0;
        for (int p = 0; p < parts; ++p) s += P[(int64_t)p * I * J + t];
        double* c = C + i + j * ldc;
        *c = alpha * s + (beta == 0.0 ? 0.0 : beta * *c);
    }
}

int g_sms = 0;

int sm_count() {
    if (!g_sms) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            g_sms = 148;
    }
    return g_sms;
}

}  // namespace

// C (I x J, column-major, ldc) = alpha X^T Y + beta C with X: K x I and Y:
// K x J row-major (ldx, ldy). The workspace of the split parts belongs to
// the context (grown on demand, reused).
int ozaki_gemm_tn(nm_ctx* ctx, cudaStream_t s, int64_t I, int64_t J, int64_t K, double alpha, const double* X,
                  int64_t ldx, const double* Y, int64_t ldy, double beta, double* C, int64_t ldc) {
    if (I <= 0 || J <= 0) return NM_OK;
    const int64_t ti = (I + kTileI - 1) / kTileI, tj = (J + kTileJ - 1) / kTileJ;
    const int64_t chunks = std::max<int64_t>((K + kChunk - 1) / kChunk, 1);
    // about four CTAs per SM in all, at least 8 chunks per part
    int64_t parts = std::max<int64_t>(1, std::min<int64_t>(chunks / 8, (4 * sm_count()) / (ti * tj)));
    parts = std::min<int64_t>(parts, 65535);
    const int64_t per = ((chunks + parts - 1) / parts) * kChunk;
    parts = (K + per - 1) / per;
    if (parts < 1) parts = 1;
    const size_t need = (size_t)parts * I * J * sizeof(double);
    if (ctx->gemm_ws.bytes < need) NM_TRY(ctx->gemm_ws.alloc(need));
    Shape sh{X, ldx, Y, ldy, I, J, K, per, ctx->gemm_ws.as<double>(), nullptr, 0, 1.0, 0.0};
    dim3 grid((unsigned)ti, (unsigned)tj, (unsigned)parts);
    if (K > 0) {
        ozaki_kernel<true, false, false><<<grid, kThreads, 0, s>>>(sh);
        count_launch();
        NM_CUDA(cudaGetLastError());
    } else {
        NM_CUDA(cudaMemsetAsync(ctx->gemm_ws.p, 0, need, s));
    }
    const int64_t tot = I * J;
    ozaki_reduce_kernel<<<(unsigned)std::min<int64_t>((tot + 255) / 256, 4096), 256, 0, s>>>(
        I, J, (int)parts, ctx->gemm_ws.as<double>(), alpha, beta, C, ldc);
    count_launch();
    NM_CUDA(cudaGetLastError());
    return NM_OK;
}

// D (I x J, row-major, ldd) = alpha X Y + beta D with X: I x K row-major
// (ldx) and Y: K x J column-major (ldy).
int ozaki_gemm_nn(cudaStream_t s, int64_t I, int64_t J, int64_t K, double alpha, const double* X, int64_t ldx,
                  const double* Y, int64_t ldy, double beta, double* D, int64_t ldd) {
    if (I <= 0 || J <= 0) return NM_OK;
    const int64_t ti = (I + kTileI - 1) / kTileI, tj = (J + kTileJ - 1) / kTileJ;
    if (ti > 0x7FFFFFFF || tj > 65535) return fail(NM_EINVAL, "product too large for one launch");
    Shape sh{X, ldx, Y, ldy, I, J, K, std::max<int64_t>(K, 1), nullptr, D, ldd, alpha, beta};
    dim3 grid((unsigned)ti, (unsigned)tj, 1);
    ozaki_kernel<false, true, true><<<grid, kThreads, 0, s>>>(sh);
    count_launch();
    NM_CUDA(cudaGetLastError());
    return NM_OK;
}

}  // namespace nm
