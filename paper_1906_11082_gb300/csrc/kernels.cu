// Hot-path sparse kernels for sm_103a.
//
// Data layout: a block of b vectors over the displacement dofs is a
// row-major (n x b) array with a leading dimension; dof 3*i + k of node i
// lives in row 3*i + k, so one node's 3 x b values are three runs of b
// consecutive entries. Each node row of a sparse matrix is handled by a
// group of TPR = min(32, next_pow2(b)) threads; thread `lane` of the group
// owns the columns lane, lane + TPR (b <= 64) and all components of them.
// A gather of a neighbour node therefore reads 3 coalesced runs of b
// values per stored block, and the matrix values and column index are
// broadcast to the group.
#include "kernels.h"

#include <atomic>
#include <cstdio>
#include <type_traits>

#include "nm_internal.h"

namespace nm {

static std::atomic<uint64_t> g_launches{0};
void count_launch(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
uint64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

static inline int tpr_shift_for(int b) {
    int t = b < 32 ? b : 32;
    int s = 0;
    while ((1 << s) < t) ++s;
    return s;
}

constexpr int kThreads = 256;

// ----------------------------------------------------------------- A (x) I_R
// Output stage shared by the plain and the tiled kernels: acc holds
// (A (x) I_R) x_k for node `row`, column c.
template <typename T, int R, int MODE>
__device__ __forceinline__ void kron_epilogue(const KronArgs<T>& a, int64_t row, int c, const T* acc) {
    if (MODE == KRON_PLAIN) {
#pragma unroll
        for (int k = 0; k < R; ++k) a.Y[(R * row + k) * a.ldy + c] = acc[k];
    } else if (MODE == KRON_CORI) {
#pragma unroll
        for (int m = 0; m < R; ++m) {
            T y = T(0);
#pragma unroll
            for (int k = 0; k < R; ++k) y += a.sk[m * 3 + k] * acc[k];
            a.Y[(R * row + m) * a.ldy + c] = y;
        }
    } else {
        const T d = a.dinv[row] * a.inv_theta;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int64_t r = R * row + k;
            const T xk = a.X[r * a.ldx + c];
            const T w = a.W[r * a.ldw + c];
            const T xp = a.Xp ? a.Xp[r * a.ldp + c] : T(0);
            const T xn = xp + a.om * (xk - xp + d * (w - acc[k]));
            if (MODE == KRON_CHEB) {
                a.Xn[r * a.ldn + c] = xn;
            } else {
                const T tk = a.Tk[r * a.ldtk + c];
                const T tp = a.Tp ? a.Tp[r * a.ldtp + c] : T(0);
                const T tn = a.a1 * (xn - a.cshift * tk) - a.a2 * tp;
                a.Tn[r * a.ldtn + c] = tn;
                if (a.Z) a.Z[r * a.ldz + c] += (a.gam_tab ? (T)a.gam_tab[c / a.gam_group] : a.gam) * tn;
            }
        }
    }
}

template <typename T, int R, int CPT, int MODE>
__global__ void __launch_bounds__(kThreads) kron_kernel(const KronArgs<T> a, int tpr_shift) {
    const int tpr = 1 << tpr_shift;
    const int lane = threadIdx.x & (tpr - 1);
    const int64_t row = (int64_t)blockIdx.x * (kThreads >> tpr_shift) + (threadIdx.x >> tpr_shift);
    if (row >= a.nrows) return;
    T acc[CPT][R];
#pragma unroll
    for (int q = 0; q < CPT; ++q)
#pragma unroll
        for (int k = 0; k < R; ++k) acc[q][k] = T(0);
    const int e0 = __ldg(a.rowptr + row), e1 = __ldg(a.rowptr + row + 1);
    for (int e = e0; e < e1; ++e) {
        const int64_t j = __ldg(a.col + e);
        const T v = __ldg(a.val + e);
        const T* xj = a.X + (int64_t)R * j * a.ldx;
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            const int c = lane + q * tpr;
            if (c < a.b) {
#pragma unroll
                for (int k = 0; k < R; ++k) acc[q][k] += v * __ldg(xj + k * a.ldx + c);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
        const int c = lane + q * tpr;
        if (c >= a.b) continue;
        kron_epilogue<T, R, MODE>(a, row, c, acc[q]);
    }
}

template <typename T, int R, int MODE>
static int kron_dispatch_cpt(int cpt, const KronArgs<T>& a, int shift, cudaStream_t s) {
    const int rows_per_block = kThreads >> shift;
    const int64_t grid = (a.nrows + rows_per_block - 1) / rows_per_block;
    if (grid == 0) return NM_OK;
    if (cpt == 1)
        kron_kernel<T, R, 1, MODE><<<(unsigned)grid, kThreads, 0, s>>>(a, shift);
    else
        kron_kernel<T, R, 2, MODE><<<(unsigned)grid, kThreads, 0, s>>>(a, shift);
    count_launch();
    NM_CUDA(cudaGetLastError());
    return NM_OK;
}

// Tiled variant for float blocks of exactly 32 columns (ld 32): one CTA per
// tile of consecutive rows. The tile's distinct neighbour nodes (R x 32
// floats each, 16-byte aligned runs) are copied into shared memory with
// cp.async; each warp then owns rows of the tile, lane = column, and reads
// its 32 (value, local column) pairs per round with one coalesced load plus
// warp shuffles.
template <int R, int MODE>
__global__ void __launch_bounds__(kThreads) kron_tile_kernel(const KronArgs<float> a) {
    extern __shared__ float4 kron_smem4[];
    float* xs = reinterpret_cast<float*>(kron_smem4);
    constexpr int RB = R * 32;          // floats per staged node
    constexpr int PER = RB / 4;         // 16-byte chunks per staged node
    const int64_t t = blockIdx.x;
    const int u0 = __ldg(a.tile_uptr + t);
    const int U = __ldg(a.tile_uptr + t + 1) - u0;
    for (int i = threadIdx.x; i < U * PER; i += kThreads) {
        const int u = i / PER, q = i - u * PER;
        const int64_t node = __ldg(a.tile_ucol + u0 + u);
        const int k = (4 * q) >> 5, cc = (4 * q) & 31;
        const float* src = a.X + ((int64_t)R * node + k) * 32 + cc;
        const unsigned dst = (unsigned)__cvta_generic_to_shared(xs + u * RB + 4 * q);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int rr = warp; rr < a.tile_rows; rr += kThreads / 32) {
        const int64_t row = t * a.tile_rows + rr;
        if (row >= a.nrows) break;
        float acc[R];
#pragma unroll
        for (int k = 0; k < R; ++k) acc[k] = 0.f;
        const int e0 = __ldg(a.rowptr + row), e1 = __ldg(a.rowptr + row + 1);
        for (int base = e0; base < e1; base += 32) {
            const int e = base + lane;
            const float vr = e < e1 ? __ldg(a.val + e) : 0.f;
            const int lr = e < e1 ? (int)__ldg(a.lcol + e) : 0;
            const int cnt = min(32, e1 - base);
            for (int j = 0; j < cnt; ++j) {
                const float v = __shfl_sync(0xffffffffu, vr, j);
                const int l = __shfl_sync(0xffffffffu, lr, j);
                const float* xr = xs + l * RB;
#pragma unroll
                for (int k = 0; k < R; ++k) acc[k] += v * xr[k * 32 + lane];
            }
        }
        kron_epilogue<float, R, MODE>(a, row, lane, acc);
    }
}

// Second tiled variant: 512 threads (16 warps) per CTA, the (value, local
// column) pairs of a round consumed four at a time with two accumulator
// sets, so each warp keeps eight shared-memory loads in flight.
template <int R, int MODE>
__global__ void __launch_bounds__(512) kron_tile2_kernel(const KronArgs<float> a) {
    extern __shared__ float4 kron_smem4[];
    float* xs = reinterpret_cast<float*>(kron_smem4);
    constexpr int RB = R * 32;
    constexpr int PER = RB / 4;
    constexpr int NT = 512;
    const int64_t t = blockIdx.x;
    const int u0 = __ldg(a.tile_uptr + t);
    const int U = __ldg(a.tile_uptr + t + 1) - u0;
    for (int i = threadIdx.x; i < U * PER; i += NT) {
        const int u = i / PER, q = i - u * PER;
        const int64_t node = __ldg(a.tile_ucol + u0 + u);
        const int k = (4 * q) >> 5, cc = (4 * q) & 31;
        const float* src = a.X + ((int64_t)R * node + k) * 32 + cc;
        const unsigned dst = (unsigned)__cvta_generic_to_shared(xs + u * RB + 4 * q);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int rr = warp; rr < a.tile_rows; rr += NT / 32) {
        const int64_t row = t * a.tile_rows + rr;
        if (row >= a.nrows) break;
        float acc[R], acc2[R];
#pragma unroll
        for (int k = 0; k < R; ++k) acc[k] = acc2[k] = 0.f;
        const int e0 = __ldg(a.rowptr + row), e1 = __ldg(a.rowptr + row + 1);
        for (int base = e0; base < e1; base += 32) {
            const int e = base + lane;
            const float vr = e < e1 ? __ldg(a.val + e) : 0.f;
            const int lr = e < e1 ? (int)__ldg(a.lcol + e) : 0;
            const int cnt = min(32, e1 - base);
            int j = 0;
            for (; j + 4 <= cnt; j += 4) {
                const float v0 = __shfl_sync(0xffffffffu, vr, j), v1 = __shfl_sync(0xffffffffu, vr, j + 1);
                const float v2 = __shfl_sync(0xffffffffu, vr, j + 2), v3 = __shfl_sync(0xffffffffu, vr, j + 3);
                const float* x0 = xs + __shfl_sync(0xffffffffu, lr, j) * RB + lane;
                const float* x1 = xs + __shfl_sync(0xffffffffu, lr, j + 1) * RB + lane;
                const float* x2 = xs + __shfl_sync(0xffffffffu, lr, j + 2) * RB + lane;
                const float* x3 = xs + __shfl_sync(0xffffffffu, lr, j + 3) * RB + lane;
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    const float a0 = x0[32 * k], a1 = x1[32 * k], a2 = x2[32 * k], a3 = x3[32 * k];
                    acc[k] = fmaf(v0, a0, acc[k]);
                    acc2[k] = fmaf(v1, a1, acc2[k]);
                    acc[k] = fmaf(v2, a2, acc[k]);
                    acc2[k] = fmaf(v3, a3, acc2[k]);
                }
            }
            for (; j < cnt; ++j) {
                const float v = __shfl_sync(0xffffffffu, vr, j);
                const float* x = xs + __shfl_sync(0xffffffffu, lr, j) * RB + lane;
#pragma unroll
                for (int k = 0; k < R; ++k) acc[k] = fmaf(v, x[32 * k], acc[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < R; ++k) acc[k] += acc2[k];
        kron_epilogue<float, R, MODE>(a, row, lane, acc);
    }
}

template <int R, int MODE>
static int kron_tile_launch(const KronArgs<float>& a, cudaStream_t s) {
    const size_t smem = (size_t)a.tile_umax * R * 32 * sizeof(float);
    static bool attr_set = false;
    if (!attr_set) {
        NM_CUDA(cudaFuncSetAttribute(kron_tile_kernel<R, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     200 * 1024));
        NM_CUDA(cudaFuncSetAttribute(kron_tile2_kernel<R, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     200 * 1024));
        attr_set = true;
    }
    if (a.tile_kernel == 2)
        kron_tile2_kernel<R, MODE><<<(unsigned)a.ntiles, 512, smem, s>>>(a);
    else
        kron_tile_kernel<R, MODE><<<(unsigned)a.ntiles, kThreads, smem, s>>>(a);
    count_launch();
    NM_CUDA(cudaGetLastError());
    return NM_OK;
}

// SM-local persistent variant for full-warp groups (b = 32 or 64): the rows
// are split into nreg contiguous regions (one per SM); each CTA reads its SM
// id and takes groups of 8 consecutive rows of that SM's region from a
// region counter, then moves on to the following regions (so every row is
// done even if some SM runs no CTA). All CTAs resident on an SM therefore
// walk adjacent Morton-ordered rows and share their neighbours in L1. The
// (value, column) pairs of a row are read 32 at a time by the warp and
// broadcast with shuffles.
template <typename T, int R, int CPT, int MODE>
__global__ void __launch_bounds__(kThreads) kron_sm_kernel(const KronArgs<T> a) {
    __shared__ int sh_group;
    unsigned smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    constexpr int GROUP = kThreads / 32;
    const int64_t N = a.nrows;
    for (int k = 0; k < a.nreg; ++k) {
        const int reg = (int)((smid + k) % (unsigned)a.nreg);
        const int64_t r0 = N * reg / a.nreg, r1 = N * (reg + 1) / a.nreg;
        const int64_t ngroups = (r1 - r0 + GROUP - 1) / GROUP;
        for (;;) {
            __syncthreads();
            if (threadIdx.x == 0) sh_group = atomicAdd(a.sched + reg, 1);
            __syncthreads();
            const int64_t g = sh_group;
            if (g >= ngroups) break;
            const int64_t row = r0 + g * GROUP + warp;
            if (row >= r1) continue;
            T acc[CPT][R];
#pragma unroll
            for (int q = 0; q < CPT; ++q)
#pragma unroll
                for (int kk = 0; kk < R; ++kk) acc[q][kk] = T(0);
            const int e0 = __ldg(a.rowptr + row), e1 = __ldg(a.rowptr + row + 1);
            for (int base = e0; base < e1; base += 32) {
                const int e = base + lane;
                const T vr = e < e1 ? __ldg(a.val + e) : T(0);
                const int cr = e < e1 ? __ldg(a.col + e) : 0;
                const int cnt = min(32, e1 - base);
                for (int jj = 0; jj < cnt; ++jj) {
                    const T v = __shfl_sync(0xffffffffu, vr, jj);
                    const int64_t j = __shfl_sync(0xffffffffu, cr, jj);
                    const T* xj = a.X + (int64_t)R * j * a.ldx;
#pragma unroll
                    for (int q = 0; q < CPT; ++q) {
                        const int c = lane + 32 * q;
                        if (c < a.b) {
#pragma unroll
                            for (int kk = 0; kk < R; ++kk) acc[q][kk] += v * __ldg(xj + kk * a.ldx + c);
                        }
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < CPT; ++q) {
                const int c = lane + 32 * q;
                if (c < a.b) kron_epilogue<T, R, MODE>(a, row, c, acc[q]);
            }
        }
    }
}

template <typename T, int R, int MODE>
static int kron_sm_launch(const KronArgs<T>& a, cudaStream_t s) {
    static int grid[2] = {0, 0};
    const int cpt = a.b > 32 ? 2 : 1;
    if (grid[cpt - 1] == 0) {
        int dev = 0, sms = 0, per = 0;
        NM_CUDA(cudaGetDevice(&dev));
        NM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        if (cpt == 1)
            NM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kron_sm_kernel<T, R, 1, MODE>, kThreads, 0));
        else
            NM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kron_sm_kernel<T, R, 2, MODE>, kThreads, 0));
        grid[cpt - 1] = sms * (per > 0 ? per : 1);
    }
    NM_CUDA(cudaMemsetAsync(a.sched, 0, a.nreg * sizeof(int), s));
    if (cpt == 1)
        kron_sm_kernel<T, R, 1, MODE><<<grid[0], kThreads, 0, s>>>(a);
    else
        kron_sm_kernel<T, R, 2, MODE><<<grid[1], kThreads, 0, s>>>(a);
    count_launch();
    NM_CUDA(cudaGetLastError());
    return NM_OK;
}

// Warp-per-row variant for blocks 17..64 wide (plain grid, 8 rows per
// CTA): the row's (value, column) pairs are read 32 at a time and consumed
// four at a time, so each lane keeps 4 R independent gathers in flight and
// two accumulator sets break the FMA chains.
template <typename T, int R, int CPT, int MODE>
__device__ __forceinline__ void warp_row(const KronArgs<T>& a, const int64_t row, const int lane) {
    T acc[CPT][R], acc2[CPT][R];
#pragma unroll
    for (int q = 0; q < CPT; ++q)
#pragma unroll
        for (int k = 0; k < R; ++k) acc[q][k] = acc2[q][k] = T(0);
    const int e0 = __ldg(a.rowptr + row), e1 = __ldg(a.rowptr + row + 1);
    const int64_t RL = (int64_t)R * a.ldx;
    for (int base = e0; base < e1; base += 32) {
        const int e = base + lane;
        const T vr = e < e1 ? __ldg(a.val + e) : T(0);
        const int cr = e < e1 ? __ldg(a.col + e) : 0;
        const int cnt = min(32, e1 - base);
        int jj = 0;
        for (; jj + 4 <= cnt; jj += 4) {
            T v[4];
            const T* x[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                v[u] = __shfl_sync(0xffffffffu, vr, jj + u);
                x[u] = a.X + RL * __shfl_sync(0xffffffffu, cr, jj + u);
            }
#pragma unroll
            for (int q = 0; q < CPT; ++q) {
                const int c = lane + 32 * q;
                if (c < a.b) {
                    T g[4][R];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int k = 0; k < R; ++k) g[u][k] = __ldg(x[u] + k * a.ldx + c);
#pragma unroll
                    for (int k = 0; k < R; ++k) {
                        acc[q][k] += v[0] * g[0][k];
                        acc2[q][k] += v[1] * g[1][k];
                        acc[q][k] += v[2] * g[2][k];
                        acc2[q][k] += v[3] * g[3][k];
                    }
                }
            }
        }
        for (; jj < cnt; ++jj) {
            const T v = __shfl_sync(0xffffffffu, vr, jj);
            const T* xj = a.X + RL * __shfl_sync(0xffffffffu, cr, jj);
#pragma unroll
            for (int q = 0; q < CPT; ++q) {
                const int c = lane + 32 * q;
                if (c < a.b) {
#pragma unroll
                    for (int k = 0; k < R; ++k) acc[q][k] += v * __ldg(xj + k * a.ldx + c);
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
        const int c = lane + 32 * q;
        if (c >= a.b) continue;
#pragma unroll
        for (int k = 0; k < R; ++k) acc[q][k] += acc2[q][k];
        kron_epilogue<T, R, MODE>(a, row, c, acc[q]);
    }
}


template <typename T, int R, int CPT, int MODE>
__global__ void __launch_bounds__(kThreads) kron_warp_kernel(const KronArgs<T> a) {
    const int lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
    if (row >= a.nrows) return;
    warp_row<T, R, CPT, MODE>(a, row, lane);
}

// Chunked warp-per-row variant: CTA c owns the contiguous row range
// [N c / G, N (c + 1) / G) of the Morton-ordered rows and its warps sweep
// it together (warp w takes rows r0 + w, r0 + w + W, ...), so the
// neighbour records of consecutive windows of W rows are re-read from L1
// instead of L2. One wave: G = SMs x resident CTAs, L1 preferred over
// shared memory.
template <typename T, int R, int CPT, int MODE>
__global__ void __launch_bounds__(1024) kron_chunk_kernel(const KronArgs<T> a) {
    const int lane = threadIdx.x & 31;
    const int W = blockDim.x >> 5;
    const int64_t r0 = (int64_t)a.nrows * blockIdx.x / gridDim.x;
    const int64_t r1 = (int64_t)a.nrows * (blockIdx.x + 1) / gridDim.x;
    for (int64_t row = r0 + (threadIdx.x >> 5); row < r1; row += W) warp_row<T, R, CPT, MODE>(a, row, lane);
}

// Vectorised warp-per-row variant for float blocks exactly 32 columns wide
// and stored densely (ldx = 32, 16-byte aligned), the width of the
// benchmark's Lanczos block. The warp splits into four groups of eight
// lanes; group g takes the row's stored entries g, g + 4, g + 8, ... and
// lane q of the group reads columns 4q..4q+3 of the R components of that
// neighbour with R 16-byte loads, so one group fetches a whole neighbour
// record (R x 32 floats) in R instructions and all 32 lanes stay busy.
// Two entries per group are in flight per trip. The four partial sums are
// combined by butterfly shuffles and lane c then takes column c for the
// shared epilogue.
template <int R, int MODE, int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) kron_v4_kernel(const KronArgs<float> a) {
    const int lane = threadIdx.x & 31;
    const int g = lane >> 3, q = lane & 7;
    int64_t blk = blockIdx.x;
    if (a.sched) {
        // SM-local order: the CTA takes the next row block of its SM's own
        // contiguous region (then of the following regions once that is
        // used up), so the CTAs resident on one SM work on neighbouring
        // Morton rows and share their gathered records in L1. The grid has
        // exactly one CTA per row block, so every block is taken once.
        __shared__ int64_t s_blk;
        if (threadIdx.x == 0) {
            unsigned smid;
            asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
            const int64_t nblk = gridDim.x;
            s_blk = -1;
            for (int k = 0; k < a.nreg; ++k) {
                const int reg = (int)((smid + k) % (unsigned)a.nreg);
                const int64_t b0 = nblk * reg / a.nreg, b1 = nblk * (reg + 1) / a.nreg;
                const int64_t take = atomicAdd(a.sched + reg, 1);
                if (take < b1 - b0) {
                    s_blk = b0 + take;
                    break;
                }
            }
        }
        __syncthreads();
        blk = s_blk;
        if (blk < 0) return;
    }
    const int64_t row = blk * (NT / 32) + (threadIdx.x >> 5);
    if (row >= a.nrows) return;
    float4 acc[R];
#pragma unroll
    for (int k = 0; k < R; ++k) acc[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    const int e0 = __ldg(a.rowptr + row), e1 = __ldg(a.rowptr + row + 1);
    // The semi-iteration epilogue's own-row operands do not depend on the
    // gather: issue their loads now so their DRAM latency overlaps it.
    constexpr bool kCheb = MODE == KRON_CHEB || MODE == KRON_CHEB_FILT;
    float pw[R], pxk[R], pxp[R], ptk[R], ptp[R];
    float pd = 0.f;
    if (kCheb) {
        pd = a.dinv[row];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int64_t r = R * row + k;
            // streamed once per step: evict-first, so the gathered block
            // keeps its L2 lines
            pxk[k] = a.X[r * a.ldx + lane];
            pw[k] = __ldcs(a.W + r * a.ldw + lane);
            pxp[k] = a.Xp ? __ldcs(a.Xp + r * a.ldp + lane) : 0.f;
            if (MODE == KRON_CHEB_FILT) {
                ptk[k] = __ldcs(a.Tk + r * a.ldtk + lane);
                ptp[k] = a.Tp ? __ldcs(a.Tp + r * a.ldtp + lane) : 0.f;
            }
        }
    }
    const float4* xb = reinterpret_cast<const float4*>(a.X) + q;
    // entries per group in flight: a 1-component record is a quarter of a
    // 3-component one, so it takes twice as many to keep the loads busy
    constexpr int U = R == 1 ? 4 : 2;
    int e = e0 + g;
    for (; e + 4 * (U - 1) < e1; e += 4 * U) {
        int j[U];
        float v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            j[u] = __ldg(a.col + e + 4 * u);
            v[u] = __ldg(a.val + e + 4 * u);
        }
        float4 x[U][R];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int k = 0; k < R; ++k) x[u][k] = __ldg(xb + (int64_t)j[u] * (8 * R) + 8 * k);
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int k = 0; k < R; ++k) {
                acc[k].x += v[u] * x[u][k].x;
                acc[k].y += v[u] * x[u][k].y;
                acc[k].z += v[u] * x[u][k].z;
                acc[k].w += v[u] * x[u][k].w;
            }
    }
    for (; e < e1; e += 4) {
        const int j0 = __ldg(a.col + e);
        const float v0 = __ldg(a.val + e);
        const float4* p0 = xb + (int64_t)j0 * (8 * R);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const float4 x0 = __ldg(p0 + 8 * k);
            acc[k].x += v0 * x0.x;
            acc[k].y += v0 * x0.y;
            acc[k].z += v0 * x0.z;
            acc[k].w += v0 * x0.w;
        }
    }
    // lanes q, q + 8, q + 16, q + 24 hold partial sums of the same columns
#pragma unroll
    for (int k = 0; k < R; ++k) {
#pragma unroll
        for (int m = 8; m <= 16; m *= 2) {
            acc[k].x += __shfl_xor_sync(0xffffffffu, acc[k].x, m);
            acc[k].y += __shfl_xor_sync(0xffffffffu, acc[k].y, m);
            acc[k].z += __shfl_xor_sync(0xffffffffu, acc[k].z, m);
            acc[k].w += __shfl_xor_sync(0xffffffffu, acc[k].w, m);
        }
    }
    // column c = lane lives in element (c & 3) of lane c >> 2
    const int src = lane >> 2, sel = lane & 3;
    float out[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const float t0 = __shfl_sync(0xffffffffu, acc[k].x, src);
        const float t1 = __shfl_sync(0xffffffffu, acc[k].y, src);
        const float t2 = __shfl_sync(0xffffffffu, acc[k].z, src);
        const float t3 = __shfl_sync(0xffffffffu, acc[k].w, src);
        out[k] = sel == 0 ? t0 : (sel == 1 ? t1 : (sel == 2 ? t2 : t3));
    }
    if (!kCheb) {
        kron_epilogue<float, R, MODE>(a, row, lane, out);
        return;
    }
    // same arithmetic as kron_epilogue, on the preloaded operands
    const float d = pd * a.inv_theta;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int64_t r = R * row + k;
        const float xn = pxp[k] + a.om * (pxk[k] - pxp[k] + d * (pw[k] - out[k]));
        if (MODE == KRON_CHEB) {
            a.Xn[r * a.ldn + lane] = xn;
        } else {
            const float tn = a.a1 * (xn - a.cshift * ptk[k]) - a.a2 * ptp[k];
            a.Tn[r * a.ldtn + lane] = tn;
            if (a.Z) a.Z[r * a.ldz + lane] += (a.gam_tab ? (float)a.gam_tab[lane / a.gam_group] : a.gam) * tn;
        }
    }
}

template <int R, int MODE>
static int kron_v4_launch(const KronArgs<float>& a, cudaStream_t s) {
    // one row per warp; larger CTAs keep more consecutive (Morton-near)
    // rows, whose neighbour sets overlap, on one SM's L1
    const int nt = R == 1 ? a.vec_threads_p : a.vec_threads;
    const int64_t grid = (a.nrows + nt / 32 - 1) / (nt / 32);
    if (grid == 0) return NM_OK;
    if (a.sched) NM_CUDA(cudaMemsetAsync(a.sched, 0, a.nreg * sizeof(int), s));
    switch (nt) {
        case 32: kron_v4_kernel<R, MODE, 32><<<(unsigned)grid, 32, 0, s>>>(a); break;
        case 64: kron_v4_kernel<R, MODE, 64><<<(unsigned)grid, 64, 0, s>>>(a); break;
        case 128: kron_v4_kernel<R, MODE, 128><<<(unsigned)grid, 128, 0, s>>>(a); break;
        case 512: kron_v4_kernel<R, MODE, 512><<<(unsigned)grid, 512, 0, s>>>(a); break;
        case 1024: kron_v4_kernel<R, MODE, 1024><<<(unsigned)grid, 1024, 0, s>>>(a); break;
        default: kron_v4_kernel<R, MODE, 256><<<(unsigned)grid, 256, 0, s>>>(a); break;
    }
    count_launch();
    NM_CUDA(cudaGetLastError());
    return NM_OK;
}

template <typename T>
static bool v4_ok(const KronArgs<T>& a) {
    return std::is_same<T, float>::value && a.vec && a.b == 32 && a.ldx == 32 && ((uintptr_t)a.X & 15) == 0;
}

template <typename T, int R, int CPT, int MODE>
static int kron_chunk_launch_t(const KronArgs<T>& a, cudaStream_t s) {
    // grid per (instantiation, CTA size), found once per process
    static int grid[3] = {0, 0, 0};
    const int nt = a.chunk;
    const int slot = nt == 256 ? 0 : (nt == 512 ? 1 : 2);
    if (grid[slot] == 0) {
        int dev = 0, sms = 0, per = 0;
        NM_CUDA(cudaGetDevice(&dev));
        NM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        NM_CUDA(cudaFuncSetAttribute(kron_chunk_kernel<T, R, CPT, MODE>,
                                     cudaFuncAttributePreferredSharedMemoryCarveout, 0));
        NM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kron_chunk_kernel<T, R, CPT, MODE>, nt, 0));
        grid[slot] = sms * (per > 0 ? per : 1);
    }
    kron_chunk_kernel<T, R, CPT, MODE><<<(unsigned)grid[slot], (unsigned)nt, 0, s>>>(a);
    count_launch();
    NM_CUDA(cudaGetLastError());
    return NM_OK;
}

template <typename T, int R, int MODE>
static int kron_chunk_launch(const KronArgs<T>& a, cudaStream_t s) {
    if (a.nrows == 0) return NM_OK;
    return a.b > 32 ? kron_chunk_launch_t<T, R, 2, MODE>(a, s) : kron_chunk_launch_t<T, R, 1, MODE>(a, s);
}

template <typename T, int R, int MODE>
static int kron_warp_launch(const KronArgs<T>& a, cudaStream_t s) {
    const int64_t grid = (a.nrows + kThreads / 32 - 1) / (kThreads / 32);
    if (grid == 0) return NM_OK;
    if (a.b > 32)
        kron_warp_kernel<T, R, 2, MODE><<<(unsigned)grid, kThreads, 0, s>>>(a);
    else
        kron_warp_kernel<T, R, 1, MODE><<<(unsigned)grid, kThreads, 0, s>>>(a);
    count_launch();
    NM_CUDA(cudaGetLastError());
    return NM_OK;
}

template <typename T>
static bool tiled_ok(const KronArgs<T>& a) {
    if (!std::is_same<T, float>::value || !a.tile_uptr || a.ntiles == 0 || a.b != 32 || a.ldx != 32) return false;
    if (((uintptr_t)a.X & 15) != 0) return false;
    return (size_t)a.tile_umax * 3 * 32 * sizeof(float) <= 200 * 1024;
}

template <typename T>
int launch_kron(int R, int mode, const KronArgs<T>& a, cudaStream_t s) {
    if (a.b < 1 || a.b > 64) return fail(NM_EINVAL, "block width must be in 1..64");
    if constexpr (std::is_same<T, float>::value) {
        if (a.tma.ntiles > 0 && R == 3 && mode == KRON_CHEB && a.b == 32 && a.ldx == 32 && !a.chunk && !a.sched)
            return launch_kron_tma(a, s);
        if (v4_ok(a) && !a.chunk) {
            if (R == 3) {
                switch (mode) {
                    case KRON_PLAIN: return kron_v4_launch<3, KRON_PLAIN>(a, s);
                    case KRON_CHEB: return kron_v4_launch<3, KRON_CHEB>(a, s);
                    case KRON_CHEB_FILT: return kron_v4_launch<3, KRON_CHEB_FILT>(a, s);
                    case KRON_CORI: return kron_v4_launch<3, KRON_CORI>(a, s);
                }
            } else if (R == 1 && mode == KRON_CHEB) {
                return kron_v4_launch<1, KRON_CHEB>(a, s);
            }
        }
    }
    if (a.sched && a.nreg > 0 && a.b >= 17 && a.b <= 64) {
        if (R == 3) {
            switch (mode) {
                case KRON_PLAIN: return kron_sm_launch<T, 3, KRON_PLAIN>(a, s);
                case KRON_CHEB: return kron_sm_launch<T, 3, KRON_CHEB>(a, s);
                case KRON_CHEB_FILT: return kron_sm_launch<T, 3, KRON_CHEB_FILT>(a, s);
                case KRON_CORI: return kron_sm_launch<T, 3, KRON_CORI>(a, s);
            }
        } else if (R == 1 && mode == KRON_CHEB) {
            return kron_sm_launch<T, 1, KRON_CHEB>(a, s);
        }
    }
    if (a.chunk && a.b >= 17 && a.b <= 64) {
        if (R == 3) {
            switch (mode) {
                case KRON_PLAIN: return kron_chunk_launch<T, 3, KRON_PLAIN>(a, s);
                case KRON_CHEB: return kron_chunk_launch<T, 3, KRON_CHEB>(a, s);
                case KRON_CHEB_FILT: return kron_chunk_launch<T, 3, KRON_CHEB_FILT>(a, s);
                case KRON_CORI: return kron_chunk_launch<T, 3, KRON_CORI>(a, s);
            }
        } else if (R == 1 && mode == KRON_CHEB) {
            return kron_chunk_launch<T, 1, KRON_CHEB>(a, s);
        }
    }
    if constexpr (std::is_same<T, float>::value) {
        if (tiled_ok(a)) {
            if (R == 3 && mode == KRON_CHEB) return kron_tile_launch<3, KRON_CHEB>(a, s);
            if (R == 3 && mode == KRON_CHEB_FILT) return kron_tile_launch<3, KRON_CHEB_FILT>(a, s);
            if (R == 3 && mode == KRON_PLAIN) return kron_tile_launch<3, KRON_PLAIN>(a, s);
            if (R == 1 && mode == KRON_CHEB) return kron_tile_launch<1, KRON_CHEB>(a, s);
        }
    }
    if (a.b >= 17 && a.b <= 64) {
        if (R == 3) {
            switch (mode) {
                case KRON_PLAIN: return kron_warp_launch<T, 3, KRON_PLAIN>(a, s);
                case KRON_CHEB: return kron_warp_launch<T, 3, KRON_CHEB>(a, s);
                case KRON_CHEB_FILT: return kron_warp_launch<T, 3, KRON_CHEB_FILT>(a, s);
                case KRON_CORI: return kron_warp_launch<T, 3, KRON_CORI>(a, s);
            }
        } else if (R == 1 && mode == KRON_CHEB) {
            return kron_warp_launch<T, 1, KRON_CHEB>(a, s);
        }
    }
    const int shift = tpr_shift_for(a.b);
    const int cpt = (a.b + (1 << shift) - 1) >> shift;
    if (R == 3) {
        switch (mode) {
            case KRON_PLAIN: return kron_dispatch_cpt<T, 3, KRON_PLAIN>(cpt, a, shift, s);
            case KRON_CHEB: return kron_dispatch_cpt<T, 3, KRON_CHEB>(cpt, a, shift, s);
            case KRON_CHEB_FILT: return kron_dispatch_cpt<T, 3, KRON_CHEB_FILT>(cpt, a, shift, s);
            case KRON_CORI: return kron_dispatch_cpt<T, 3, KRON_CORI>(cpt, a, shift, s);
        }
    } else if (R == 1) {
        switch (mode) {
            case KRON_PLAIN: return kron_dispatch_cpt<T, 1, KRON_PLAIN>(cpt, a, shift, s);
            case KRON_CHEB: return kron_dispatch_cpt<T, 1, KRON_CHEB>(cpt, a, shift, s);
            default: break;
        }
    }
    return fail(NM_EINVAL, "unsupported kron mode");
}

// ----------------------------------------------------------------- 3x3 BSR
template <typename T, int CPT>
__global__ void __launch_bounds__(kThreads) bsr33_kernel(const Bsr33Args<T> a, int tpr_shift) {
    const int tpr = 1 << tpr_shift;
    const int lane = threadIdx.x & (tpr - 1);
    const int64_t row = (int64_t)blockIdx.x * (kThreads >> tpr_shift) + (threadIdx.x >> tpr_shift);
    if (row >= a.nrows) return;
    T acc[CPT][3];
#pragma unroll
    for (int q = 0; q < CPT; ++q) acc[q][0] = acc[q][1] = acc[q][2] = T(0);
    const int e0 = __ldg(a.rowptr + row), e1 = __ldg(a.rowptr + row + 1);
    for (int e = e0; e < e1; ++e) {
        const int64_t j = __ldg(a.col + e);
        const T* K = a.val + 9 * (int64_t)e;
        T k[9];
#pragma unroll
        for (int t = 0; t < 9; ++t) k[t] = __ldg(K + t);
        const T* xj = a.X + 3 * j * a.ldx;
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            const int c = lane + q * tpr;
            if (c < a.b) {
                const T x0 = __ldg(xj + c), x1 = __ldg(xj + a.ldx + c), x2 = __ldg(xj + 2 * a.ldx + c);
                acc[q][0] += k[0] * x0 + k[1] * x1 + k[2] * x2;
                acc[q][1] += k[3] * x0 + k[4] * x1 + k[5] * x2;
                acc[q][2] += k[6] * x0 + k[7] * x1 + k[8] * x2;
            }
        }
    }
    if (a.e_rowptr) {
        const int f0 = __ldg(a.e_rowptr + row), f1 = __ldg(a.e_rowptr + row + 1);
        for (int e = f0; e < f1; ++e) {
            const int64_t p = __ldg(a.e_col + e);
            const T v0 = __ldg(a.e_val + 3 * (int64_t)e), v1 = __ldg(a.e_val + 3 * (int64_t)e + 1),
                    v2 = __ldg(a.e_val + 3 * (int64_t)e + 2);
#pragma unroll
            for (int q = 0; q < CPT; ++q) {
                const int c = lane + q * tpr;
                if (c < a.b) {
                    const T sv = __ldg(a.S + p * a.lds + c);
                    acc[q][0] += v0 * sv;
                    acc[q][1] += v1 * sv;
                    acc[q][2] += v2 * sv;
                }
            }
        }
    }
    const T d = a.X1 ? a.dinv[row] * a.inv_theta : T(0);
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
        const int c = lane + q * tpr;
        if (c >= a.b) continue;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            a.W[(3 * row + m) * a.ldw + c] = acc[q][m];
            if (a.X1) a.X1[(3 * row + m) * a.ldx1 + c] = d * acc[q][m];
        }
    }
}

template <typename T>
int launch_bsr33(const Bsr33Args<T>& a, cudaStream_t s) {
    if (a.b < 1 || a.b > 64) return fail(NM_EINVAL, "block width must be in 1..64");
    const int shift = tpr_shift_for(a.b);
    const int cpt = (a.b + (1 << shift) - 1) >> shift;
    const int rows_per_block = kThreads >> shift;
    const int64_t grid = (a.nrows + rows_per_block - 1) / rows_per_block;
    if (grid == 0) return NM_OK;
    if (cpt == 1)
        bsr33_kernel<T, 1><<<(unsigned)grid, kThreads, 0, s>>>(a, shift);
    else
        bsr33_kernel<T, 2><<<(unsigned)grid, kThreads, 0, s>>>(a, shift);
    count_launch();
    NM_CUDA(cudaGetLastError());
    return NM_OK;
}

// ----------------------------------------------------------------- 1x3 BSR
template <typename T, int CPT>
__global__ void __launch_bounds__(kThreads) bsr13_kernel(const Bsr13Args<T> a, int tpr_shift) {
    const int tpr = 1 << tpr_shift;
    const int lane = threadIdx.x & (tpr - 1);
    const int64_t row = (int64_t)blockIdx.x * (kThreads >> tpr_shift) + (threadIdx.x >> tpr_shift);
    if (row >= a.nrows) return;
    T acc[CPT];
#pragma unroll
    for (int q = 0; q < CPT; ++q) acc[q] = T(0);
    const int e0 = __ldg(a.rowptr + row), e1 = __ldg(a.rowptr + row + 1);
    for (int e = e0; e < e1; ++e) {
        const int64_t j = __ldg(a.col + e);
        const T v0 = __ldg(a.val + 3 * (int64_t)e), v1 = __ldg(a.val + 3 * (int64_t)e + 1),
                v2 = __ldg(a.val + 3 * (int64_t)e + 2);
        const T* xj = a.X + 3 * j * a.ldx;
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            const int c = lane + q * tpr;
            if (c < a.b)
                acc[q] += v0 * __ldg(xj + c) + v1 * __ldg(xj + a.ldx + c) + v2 * __ldg(xj + 2 * a.ldx + c);
        }
    }
    const T d = a.S1 ? a.dinv[row] * a.inv_theta : T(0);
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
        const int c = lane + q * tpr;
        if (c >= a.b) continue;
        a.Q[row * a.ldq + c] = acc[q];
        if (a.S1) a.S1[row * a.lds1 + c] = d * acc[q];
    }
}

template <typename T>
int launch_bsr13(const Bsr13Args<T>& a, cudaStream_t s) {
    if (a.b < 1 || a.b > 64) return fail(NM_EINVAL, "block width must be in 1..64");
    const int shift = tpr_shift_for(a.b);
    const int cpt = (a.b + (1 << shift) - 1) >> shift;
    const int rows_per_block = kThreads >> shift;
    const int64_t grid = (a.nrows + rows_per_block - 1) / rows_per_block;
    if (grid == 0) return NM_OK;
    if (cpt == 1)
        bsr13_kernel<T, 1><<<(unsigned)grid, kThreads, 0, s>>>(a, shift);
    else
        bsr13_kernel<T, 2><<<(unsigned)grid, kThreads, 0, s>>>(a, shift);
    count_launch();
    NM_CUDA(cudaGetLastError());
    return NM_OK;
}

// ----------------------------------------------------------------- small kernels
template <typename T>
__global__ void scale_copy_kernel(int64_t rows, int b, T alpha, const T* X, int64_t ldx, T* Y,
                                  int64_t ldy) {
    const int64_t total = rows * b;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / b;
        const int c = (int)(t - i * b);
        Y[i * ldy + c] = alpha * X[i * ldx + c];
    }
}

static unsigned grid_for(int64_t total) {
    int64_t g = (total + kThreads - 1) / kThreads;
    if (g > 152 * 32) g = 152 * 32;
    if (g < 1) g = 1;
    return (unsigned)g;
}

template <typename T>
int launch_scale_copy(int64_t rows, int b, T alpha, const T* X, int64_t ldx, T* Y, int64_t ldy,
                      cudaStream_t s) {
    if (rows * b == 0) return NM_OK;
    scale_copy_kernel<T><<<grid_for(rows * b), kThreads, 0, s>>>(rows, b, alpha, X, ldx, Y, ldy);
    count_launch();
    NM_CUDA(cudaGetLastError());
    return NM_OK;
}

template <typename Tin, typename Tout>
__global__ void convert_kernel(int64_t rows, int b, const Tin* X, int64_t ldx, Tout* Y, int64_t ldy) {
    const int64_t total = rows * b;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / b;
        const int c = (int)(t - i * b);
        Y[i * ldy + c] = (Tout)X[i * ldx + c];
    }
}

// w32 = float(W) and the first semi-iteration step x1 = inv_theta D^-1 w32
// in one pass (the same float expression as dscale_kernel).
__global__ void convert_x1_kernel(int R, int64_t nodes, int b, const double* W, int64_t ldw, float* w32,
                                  float inv_theta, const float* dinv, float* x1) {
    const int64_t total = (int64_t)R * nodes * b;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / b;
        const int c = (int)(t - r * b);
        const float w = (float)W[r * ldw + c];
        w32[t] = w;
        x1[t] = inv_theta * dinv[r / R] * w;
    }
}

int launch_convert_x1(int R, int64_t nodes, int b, const double* W, int64_t ldw, float* w32, float inv_theta,
                      const float* dinv, float* x1, cudaStream_t s) {
    const int64_t total = (int64_t)R * nodes * b;
    if (total == 0) return NM_OK;
    convert_x1_kernel<<<grid_for(total), kThreads, 0, s>>>(R, nodes, b, W, ldw, w32, inv_theta, dinv, x1);
    count_launch();
    NM_CUDA(cudaGetLastError());
    return NM_OK;
}

template <typename Tin, typename Tout>
int launch_convert(int64_t rows, int b, const Tin* X, int64_t ldx, Tout* Y, int64_t ldy,
                   cudaStream_t s) {
    if (rows * b == 0) return NM_OK;
    convert_kernel<Tin, Tout><<<grid_for(rows * b), kThreads, 0, s>>>(rows, b, X, ldx, Y, ldy);
    count_launch();
    NM_CUDA(cudaGetLastError());
    return NM_OK;
}

__global__ void d2f_kernel(int64_t n, const double* x, float* y) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
         t += (int64_t)gridDim.x * blockDim.x)
        y[t] = (float)x[t];
}

int launch_d2f(int64_t n, const double* x, float* y, cudaStream_t s) {
    if (n == 0) return NM_OK;
    d2f_kernel<<<grid_for(n), kThreads, 0, s>>>(n, x, y);
    count_launch();
    NM_CUDA(cudaGetLastError());
    return NM_OK;
}

// column sums of squares: threadIdx.x over 32 columns, blocks stride over rows
__global__ void colnorm2_kernel(int64_t rows, int b, const double* X, int64_t ldx, double* out) {
    const int c = blockIdx.y * 32 + threadIdx.x;
    double s = 0.0;
    if (c < b) {
        for (int64_t i = blockIdx.x * (int64_t)blockDim.y + threadIdx.y; i < rows;
             i += (int64_t)gridDim.x * blockDim.y) {
            const double v = X[i * ldx + c];
            s += v * v;
        }
    }
    __shared__ double red[8][33];
    red[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && c < b) {
        double t = 0.0;
        for (int y = 0; y < (int)blockDim.y; ++y) t += red[y][threadIdx.x];
        atomicAdd(out + c, t);
    }
}

int launch_colnorm2(int64_t rows, int b, const double* X, int64_t ldx, double* out, cudaStream_t s) {
    if (rows == 0 || b == 0) return NM_OK;
    dim3 block(32, 8);
    int64_t gx = (rows + 8 * 64 - 1) / (8 * 64);
    if (gx > 152 * 4) gx = 152 * 4;
    dim3 grid((unsigned)gx, (unsigned)((b + 31) / 32));
    colnorm2_kernel<<<grid, block, 0, s>>>(rows, b, X, ldx, out);
    count_launch();
    NM_CUDA(cudaGetLastError());
    return NM_OK;
}

__global__ void resid_block_kernel(int64_t rows, int b, const double* KX, const double* MX,
                                   const double* lam, double* R) {
    const int64_t total = rows * b;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(t % b);
        R[t] = KX[t] - lam[c] * MX[t];
    }
}

int launch_resid_block(int64_t rows, int b, const double* KX, const double* MX, const double* lam,
                       double* R, cudaStream_t s) {
    if (rows * b == 0) return NM_OK;
    resid_block_kernel<<<grid_for(rows * b), kThreads, 0, s>>>(rows, b, KX, MX, lam, R);
    count_launch();
    NM_CUDA(cudaGetLastError());
    return NM_OK;
}

template <typename T>
__global__ void dscale_kernel(int R, int64_t nodes, int b, T inv_theta, const T* dinv, const T* W, int64_t ldw,
                              T* X, int64_t ldx) {
    const int64_t total = (int64_t)R * nodes * b;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / b;
        const int c = (int)(t - r * b);
        X[r * ldx + c] = inv_theta * dinv[r / R] * W[r * ldw + c];
    }
}

template <typename T>
int launch_dscale(int R, int64_t nodes, int b, T inv_theta, const T* dinv, const T* W, int64_t ldw, T* X,
                  int64_t ldx, cudaStream_t s) {
    const int64_t total = (int64_t)R * nodes * b;
    if (total == 0) return NM_OK;
    dscale_kernel<T><<<grid_for(total), kThreads, 0, s>>>(R, nodes, b, inv_theta, dinv, W, ldw, X, ldx);
    count_launch();
    NM_CUDA(cudaGetLastError());
    return NM_OK;
}

template <int R, int CPT>
__global__ void __launch_bounds__(kThreads) resid_mixed_kernel(int64_t nodes, const int* __restrict__ rowptr,
                                                               const int* __restrict__ col,
                                                               const double* __restrict__ val,
                                                               const double* __restrict__ W, int64_t ldw,
                                                               const float* __restrict__ x, float* r, int b,
                                                               int tpr_shift) {
    const int tpr = 1 << tpr_shift;
    const int lane = threadIdx.x & (tpr - 1);
    const int64_t row = (int64_t)blockIdx.x * (kThreads >> tpr_shift) + (threadIdx.x >> tpr_shift);
    if (row >= nodes) return;
    double acc[CPT][R];
#pragma unroll
    for (int q = 0; q < CPT; ++q)
#pragma unroll
        for (int k = 0; k < R; ++k) acc[q][k] = 0.0;
    const int e0 = __ldg(rowptr + row), e1 = __ldg(rowptr + row + 1);
    for (int e = e0; e < e1; ++e) {
        const int64_t j = __ldg(col + e);
        const double v = __ldg(val + e);
        const float* xj = x + (int64_t)R * j * b;
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            const int c = lane + q * tpr;
            if (c < b) {
#pragma unroll
                for (int k = 0; k < R; ++k) acc[q][k] += v * (double)__ldg(xj + k * b + c);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
        const int c = lane + q * tpr;
        if (c >= b) continue;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int64_t rr = R * row + k;
            r[rr * b + c] = (float)(W[rr * ldw + c] - acc[q][k]);
        }
    }
}

int launch_resid_mixed(int R, int64_t nodes, const int* rowptr, const int* col, const double* val,
                       const double* W, int64_t ldw, const float* x32, float* r32, int b, cudaStream_t s) {
    if (b < 1 || b > 64) return fail(NM_EINVAL, "block width must be in 1..64");
    const int shift = tpr_shift_for(b);
    const int cpt = (b + (1 << shift) - 1) >> shift;
    const int64_t grid = (nodes + (kThreads >> shift) - 1) / (kThreads >> shift);
    if (grid == 0) return NM_OK;
    if (R == 3 && cpt == 1)
        resid_mixed_kernel<3, 1><<<(unsigned)grid, kThreads, 0, s>>>(nodes, rowptr, col, val, W, ldw, x32, r32, b, shift);
    else if (R == 3)
        resid_mixed_kernel<3, 2><<<(unsigned)grid, kThreads, 0, s>>>(nodes, rowptr, col, val, W, ldw, x32, r32, b, shift);
    else if (cpt == 1)
        resid_mixed_kernel<1, 1><<<(unsigned)grid, kThreads, 0, s>>>(nodes, rowptr, col, val, W, ldw, x32, r32, b, shift);
    else
        resid_mixed_kernel<1, 2><<<(unsigned)grid, kThreads, 0, s>>>(nodes, rowptr, col, val, W, ldw, x32, r32, b, shift);
    count_launch();
    NM_CUDA(cudaGetLastError());
    return NM_OK;
}

__global__ void combine_kernel(const CombineArgs a) {
    const int64_t total = a.rows * a.b;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const double sv = (double)a.x32[t] + (double)a.e32[t];
        if (!a.Tn) {
            a.out[t] = sv;
            continue;
        }
        const double tp = a.Tp ? a.Tp[t] : 0.0;
        const double tn = a.a1 * (sv - a.cshift * a.Tk[t]) - a.a2 * tp;
        a.Tn[t] = tn;
        if (a.Th) {   // exact float pair of tn for the next double-float K_eff SpMM
            const float h = __double2float_rn(tn);
            a.Th[t] = h;
            a.Tl[t] = __double2float_rn(tn - (double)h);
        }
        if (a.Z) {
            const int64_t i = t / a.b;
            const int c = (int)(t - i * a.b);
            const double gm = a.deg ? a.gam_tab[(int64_t)(a.deg[0] + 1) * a.gam_stride + c / a.gam_group]
                                    : (a.gam_tab ? a.gam_tab[c / a.gam_group] : a.gam);
            a.Z[i * a.ldz + c] += gm * tn;
        }
    }
}

// W[3i + m, c] += sum_f E[f, m] S[col(f), c] for the 3x1-block CSR E over
// u-node rows (the fluid coupling of K_eff), in double; one warp per row,
// rows without entries return at once.
__global__ void bsr31_add_kernel(int nrows, const int* __restrict__ rowptr, const int* __restrict__ col,
                                 const double* __restrict__ val, const double* __restrict__ S, int64_t lds, int b,
                                 double* W, int64_t ldw) {
    const int lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
    if (row >= nrows) return;
    const int f0 = __ldg(rowptr + row), f1 = __ldg(rowptr + row + 1);
    if (f0 == f1) return;
    for (int c = lane; c < b; c += 32) {
        double acc[3] = {0.0, 0.0, 0.0};
        for (int f = f0; f < f1; ++f) {
            const double sv = __ldg(S + (int64_t)__ldg(col + f) * lds + c);
#pragma unroll
            for (int m = 0; m < 3; ++m) acc[m] += __ldg(val + 3 * (int64_t)f + m) * sv;
        }
#pragma unroll
        for (int m = 0; m < 3; ++m) W[(3 * row + m) * ldw + c] += acc[m];
    }
}

int launch_bsr31_add(int nrows, const int* rowptr, const int* col, const double* val, const double* S, int64_t lds,
                     int b, double* W, int64_t ldw, cudaStream_t s) {
    const int64_t grid = (nrows + kThreads / 32 - 1) / (kThreads / 32);
    if (grid == 0) return NM_OK;
    bsr31_add_kernel<<<(unsigned)grid, kThreads, 0, s>>>(nrows, rowptr, col, val, S, lds, b, W, ldw);
    count_launch();
    NM_CUDA(cudaGetLastError());
    return NM_OK;
}

__global__ void set_int_kernel(int* p, int v) { *p = v; }
__global__ void inc_int_kernel(int* p) { *p += 1; }

int launch_set_int(int* p, int v, cudaStream_t s) {
    set_int_kernel<<<1, 1, 0, s>>>(p, v);
    count_launch();
    NM_CUDA(cudaGetLastError());
    return NM_OK;
}

int launch_inc_int(int* p, cudaStream_t s) {
    inc_int_kernel<<<1, 1, 0, s>>>(p);
    count_launch();
    NM_CUDA(cudaGetLastError());
    return NM_OK;
}

// The same update two columns per thread (b even, operands 8/16-byte
// aligned, Z's leading dimension even, rows * b / 2 < 2^30): 32-bit index
// arithmetic, float2 / double2 accesses, identical arithmetic per element.
__global__ void combine2_kernel(const CombineArgs a) {
    const int hb = a.b >> 1;
    const int total = (int)(a.rows * hb);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const float2 x = reinterpret_cast<const float2*>(a.x32)[t];
        const float2 e = reinterpret_cast<const float2*>(a.e32)[t];
        const double s0 = (double)x.x + (double)e.x, s1 = (double)x.y + (double)e.y;
        if (!a.Tn) {
            reinterpret_cast<double2*>(a.out)[t] = make_double2(s0, s1);
            continue;
        }
        const double2 tk = reinterpret_cast<const double2*>(a.Tk)[t];
        const double2 tp = a.Tp ? reinterpret_cast<const double2*>(a.Tp)[t] : make_double2(0.0, 0.0);
        const double n0 = a.a1 * (s0 - a.cshift * tk.x) - a.a2 * tp.x;
        const double n1 = a.a1 * (s1 - a.cshift * tk.y) - a.a2 * tp.y;
        reinterpret_cast<double2*>(a.Tn)[t] = make_double2(n0, n1);
        if (a.Th) {
            const float h0 = __double2float_rn(n0), h1 = __double2float_rn(n1);
            reinterpret_cast<float2*>(a.Th)[t] = make_float2(h0, h1);
            reinterpret_cast<float2*>(a.Tl)[t] =
                make_float2(__double2float_rn(n0 - (double)h0), __double2float_rn(n1 - (double)h1));
        }
        if (a.Z) {
            const int i = t / hb;
            const int c = 2 * (t - i * hb);
            double g0, g1;
            if (a.deg) {
                const double* gt = a.gam_tab + (int64_t)(a.deg[0] + 1) * a.gam_stride;
                g0 = gt[c / a.gam_group];
                g1 = gt[(c + 1) / a.gam_group];
            } else if (a.gam_tab) {
                g0 = a.gam_tab[c / a.gam_group];
                g1 = a.gam_tab[(c + 1) / a.gam_group];
            } else {
                g0 = g1 = a.gam;
            }
            double2* zp = reinterpret_cast<double2*>(a.Z + (int64_t)i * a.ldz + c);
            double2 z = *zp;
            z.x += g0 * n0;
            z.y += g1 * n1;
            *zp = z;
        }
    }
}

int launch_combine(const CombineArgs& a, cudaStream_t s) {
    if (a.rows * a.b == 0) return NM_OK;
    const uintptr_t al16 = (uintptr_t)a.out | (uintptr_t)a.Tk | (uintptr_t)a.Tp | (uintptr_t)a.Tn | (uintptr_t)a.Z;
    const uintptr_t al8 = (uintptr_t)a.x32 | (uintptr_t)a.e32 | (uintptr_t)a.Th | (uintptr_t)a.Tl;
    if (a.b % 2 == 0 && (al16 & 15) == 0 && (al8 & 7) == 0 && (a.ldz % 2) == 0 && a.rows * a.b / 2 < (1ll << 30)) {
        combine2_kernel<<<grid_for(a.rows * a.b / 2), kThreads, 0, s>>>(a);
        count_launch();
        NM_CUDA(cudaGetLastError());
        return NM_OK;
    }
    combine_kernel<<<grid_for(a.rows * a.b), kThreads, 0, s>>>(a);
    count_launch();
    NM_CUDA(cudaGetLastError());
    return NM_OK;
}

// ----------------------------------------------------------------- double-float
// sh + sl += (ah + al)(xh + xl) to ~2^-48: TwoProduct of the leading terms by
// FMA, the cross terms by FMA, TwoSum into the leading accumulator and a
// FastTwoSum renormalisation. The _rn intrinsics keep the compiler from
// contracting or reassociating the error-free transformations.
__device__ __forceinline__ void df_fma(float& sh, float& sl, float ah, float al, float xh, float xl) {
    const float p = __fmul_rn(ah, xh);
    const float e = __fmaf_rn(ah, xh, -p);
    const float t = __fmaf_rn(ah, xl, __fmaf_rn(al, xh, e));
    const float s = __fadd_rn(sh, p);
    const float bp = __fadd_rn(s, -sh);
    const float err = __fadd_rn(__fadd_rn(sh, -__fadd_rn(s, -bp)), __fadd_rn(p, -bp));
    const float lo = __fadd_rn(__fadd_rn(sl, err), t);
    sh = __fadd_rn(s, lo);
    sl = __fadd_rn(lo, -__fadd_rn(sh, -s));
}

__global__ void split_kernel(int64_t rows, int b, const double* X, int64_t ldx, float* Xh, float* Xl) {
    const int64_t total = rows * b;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / b;
        const int c = (int)(t - i * b);
        const double x = X[i * ldx + c];
        const float h = __double2float_rn(x);
        Xh[t] = h;
        Xl[t] = __double2float_rn(x - (double)h);
    }
}

template <int CPT>
__global__ void __launch_bounds__(kThreads) bsr33_df_kernel(const Bsr33DfArgs a, int tpr_shift) {
    const int tpr = 1 << tpr_shift;
    const int lane = threadIdx.x & (tpr - 1);
    const int64_t row = (int64_t)blockIdx.x * (kThreads >> tpr_shift) + (threadIdx.x >> tpr_shift);
    if (row >= a.nrows) return;
    float sh[CPT][3], sl[CPT][3];
#pragma unroll
    for (int q = 0; q < CPT; ++q)
#pragma unroll
        for (int m = 0; m < 3; ++m) sh[q][m] = sl[q][m] = 0.f;
    const int e0 = __ldg(a.rowptr + row), e1 = __ldg(a.rowptr + row + 1);
    for (int e = e0; e < e1; ++e) {
        const int64_t j = __ldg(a.col + e);
        float kh[9], kl[9];
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            kh[t] = __ldg(a.vh + 9 * (int64_t)e + t);
            kl[t] = __ldg(a.vl + 9 * (int64_t)e + t);
        }
        const int64_t base = 3 * j * a.b;
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            const int c = lane + q * tpr;
            if (c < a.b) {
                float xh[3], xl[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    xh[k] = __ldg(a.Xh + base + k * a.b + c);
                    xl[k] = __ldg(a.Xl + base + k * a.b + c);
                }
#pragma unroll
                for (int m = 0; m < 3; ++m)
#pragma unroll
                    for (int k = 0; k < 3; ++k) df_fma(sh[q][m], sl[q][m], kh[3 * m + k], kl[3 * m + k], xh[k], xl[k]);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
        const int c = lane + q * tpr;
        if (c >= a.b) continue;
        double acc[3];
#pragma unroll
        for (int m = 0; m < 3; ++m) acc[m] = (double)sh[q][m] + (double)sl[q][m];
        if (a.e_rowptr) {
            const int f0 = __ldg(a.e_rowptr + row), f1 = __ldg(a.e_rowptr + row + 1);
            for (int e = f0; e < f1; ++e) {
                const int64_t p = __ldg(a.e_col + e);
                const double sv = __ldg(a.S + p * a.lds + c);
#pragma unroll
                for (int m = 0; m < 3; ++m) acc[m] += __ldg(a.e_val + 3 * (int64_t)e + m) * sv;
            }
        }
#pragma unroll
        for (int m = 0; m < 3; ++m) a.W[(3 * row + m) * a.ldw + c] = acc[m];
    }
}

template <int R, int CPT>
__global__ void __launch_bounds__(kThreads) resid_df_kernel(int64_t nodes, const int* __restrict__ rowptr,
                                                            const int* __restrict__ col, const float* __restrict__ vh,
                                                            const float* __restrict__ vl, const double* __restrict__ W,
                                                            int64_t ldw, const float* __restrict__ x, float* r, int b,
                                                            int tpr_shift) {
    const int tpr = 1 << tpr_shift;
    const int lane = threadIdx.x & (tpr - 1);
    const int64_t row = (int64_t)blockIdx.x * (kThreads >> tpr_shift) + (threadIdx.x >> tpr_shift);
    if (row >= nodes) return;
    float sh[CPT][R], sl[CPT][R];
#pragma unroll
    for (int q = 0; q < CPT; ++q)
#pragma unroll
        for (int k = 0; k < R; ++k) sh[q][k] = sl[q][k] = 0.f;
    const int e0 = __ldg(rowptr + row), e1 = __ldg(rowptr + row + 1);
    for (int e = e0; e < e1; ++e) {
        const int64_t j = __ldg(col + e);
        const float mh = __ldg(vh + e), ml = __ldg(vl + e);
        const float* xj = x + (int64_t)R * j * b;
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
            const int c = lane + q * tpr;
            if (c < b) {
#pragma unroll
                for (int k = 0; k < R; ++k) df_fma(sh[q][k], sl[q][k], mh, ml, __ldg(xj + k * b + c), 0.f);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
        const int c = lane + q * tpr;
        if (c >= b) continue;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const int64_t rr = R * row + k;
            r[rr * b + c] = (float)((W[rr * ldw + c] - (double)sh[q][k]) - (double)sl[q][k]);
        }
    }
}

// Dot2-style double-float accumulation (Ogita, Rump and Oishi): the
// rounding error of each product (exact via FMA), the first-order terms of
// the operands' low parts and the TwoSum error of each addition are
// collected in sl; sh carries the running float sum. sl stays ~n ulp(sh),
// so it needs no renormalisation until the final (double) sh + sl.
__device__ __forceinline__ void df_acc(float& sh, float& sl, float ah, float al, float xh, float xl) {
    const float p = __fmul_rn(ah, xh);
    const float e = __fmaf_rn(ah, xh, -p);
    const float t = __fmaf_rn(ah, xl, __fmaf_rn(al, xh, e));
    const float s = __fadd_rn(sh, p);
    const float bp = __fadd_rn(s, -sh);
    const float err = __fadd_rn(__fadd_rn(sh, -__fadd_rn(s, -bp)), __fadd_rn(p, -bp));
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(err, t));
}

// (sh, sl) += (h2, l2) for two Dot2 accumulators.
__device__ __forceinline__ void df_merge(float& sh, float& sl, float h2, float l2) {
    const float s = __fadd_rn(sh, h2);
    const float bp = __fadd_rn(s, -sh);
    const float err = __fadd_rn(__fadd_rn(sh, -__fadd_rn(s, -bp)), __fadd_rn(h2, -bp));
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(err, l2));
}

// Butterfly-combine the four lane groups' accumulators (lanes q, q + 8,
// q + 16, q + 24 hold partial sums of the same four columns).
template <int N>
__device__ __forceinline__ void df_group_reduce(float (&sh)[N], float (&sl)[N]) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int m = 8; m <= 16; m *= 2) {
            const float h2 = __shfl_xor_sync(0xffffffffu, sh[i], m);
            const float l2 = __shfl_xor_sync(0xffffffffu, sl[i], m);
            df_merge(sh[i], sl[i], h2, l2);
        }
    }
}

// W = A X (+ E S) in double-float for blocks exactly 32 wide with the split
// operand stored densely (ld 32): one warp per 3x3-block row, four groups
// of eight lanes taking every fourth stored block, lane q of a group
// holding columns 4q..4q+3 of the three output components and reading the
// neighbour's (hi, lo) records with 16-byte loads. After the groups are
// combined, group m < 3 writes output component m (and adds the pressure
// coupling in double, as the generic kernel does).
template <int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) bsr33_df_v4_kernel(const Bsr33DfArgs a) {
    const int lane = threadIdx.x & 31;
    const int g = lane >> 3, q = lane & 7;
    const int64_t row = (int64_t)blockIdx.x * (NT / 32) + (threadIdx.x >> 5);
    if (row >= a.nrows) return;
    float sh[12], sl[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) sh[i] = sl[i] = 0.f;
    const int e0 = __ldg(a.rowptr + row), e1 = __ldg(a.rowptr + row + 1);
    const float4* xh4 = reinterpret_cast<const float4*>(a.Xh) + q;
    const float4* xl4 = reinterpret_cast<const float4*>(a.Xl) + q;
    for (int e = e0 + g; e < e1; e += 4) {
        const int64_t j = __ldg(a.col + e);
        const float* kh = a.vh + 9 * (int64_t)e;
        const float* kl = a.vl + 9 * (int64_t)e;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float4 xh = __ldg(xh4 + j * 24 + 8 * k);
            const float4 xl = __ldg(xl4 + j * 24 + 8 * k);
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const float ah = __ldg(kh + 3 * m + k), al = __ldg(kl + 3 * m + k);
                df_acc(sh[4 * m + 0], sl[4 * m + 0], ah, al, xh.x, xl.x);
                df_acc(sh[4 * m + 1], sl[4 * m + 1], ah, al, xh.y, xl.y);
                df_acc(sh[4 * m + 2], sl[4 * m + 2], ah, al, xh.z, xl.z);
                df_acc(sh[4 * m + 3], sl[4 * m + 3], ah, al, xh.w, xl.w);
            }
        }
    }
    df_group_reduce<12>(sh, sl);
    if (g >= 3) return;
    const int m = g;
    double acc[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float h = m == 0 ? sh[c] : (m == 1 ? sh[4 + c] : sh[8 + c]);
        const float l = m == 0 ? sl[c] : (m == 1 ? sl[4 + c] : sl[8 + c]);
        acc[c] = (double)h + (double)l;
    }
    if (a.e_rowptr) {
        const int f0 = __ldg(a.e_rowptr + row), f1 = __ldg(a.e_rowptr + row + 1);
        for (int f = f0; f < f1; ++f) {
            const int64_t p = __ldg(a.e_col + f);
            const double ev = __ldg(a.e_val + 3 * (int64_t)f + m);
            const double* sp = a.S + p * a.lds + 4 * q;
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[c] += ev * __ldg(sp + c);
        }
    }
    double* wp = a.W + (3 * row + m) * a.ldw + 4 * q;
#pragma unroll
    for (int c = 0; c < 4; ++c) wp[c] = acc[c];
}

// r32 = float(W - (A (x) I_R) x32) for blocks exactly 32 wide (x32 and r32
// dense, ld 32), with the lane-group layout of bsr33_df_v4_kernel.
template <int R, int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) resid_df_v4_kernel(int64_t nodes, const int* __restrict__ rowptr,
                                                                  const int* __restrict__ col,
                                                                  const float* __restrict__ vh,
                                                                  const float* __restrict__ vl,
                                                                  const double* __restrict__ W, int64_t ldw,
                                                                  const float* __restrict__ x, float* r,
                                                                  const float* __restrict__ dinv, float inv_theta,
                                                                  float* x1) {
    const int lane = threadIdx.x & 31;
    const int g = lane >> 3, q = lane & 7;
    const int64_t row = (int64_t)blockIdx.x * (NT / 32) + (threadIdx.x >> 5);
    if (row >= nodes) return;
    float sh[4 * R], sl[4 * R];
#pragma unroll
    for (int i = 0; i < 4 * R; ++i) sh[i] = sl[i] = 0.f;
    const int e0 = __ldg(rowptr + row), e1 = __ldg(rowptr + row + 1);
    const float4* x4 = reinterpret_cast<const float4*>(x) + q;
    for (int e = e0 + g; e < e1; e += 4) {
        const int64_t j = __ldg(col + e);
        const float mh = __ldg(vh + e), ml = __ldg(vl + e);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const float4 xv = __ldg(x4 + j * (8 * R) + 8 * k);
            df_acc(sh[4 * k + 0], sl[4 * k + 0], mh, ml, xv.x, 0.f);
            df_acc(sh[4 * k + 1], sl[4 * k + 1], mh, ml, xv.y, 0.f);
            df_acc(sh[4 * k + 2], sl[4 * k + 2], mh, ml, xv.z, 0.f);
            df_acc(sh[4 * k + 3], sl[4 * k + 3], mh, ml, xv.w, 0.f);
        }
    }
    df_group_reduce<4 * R>(sh, sl);
    if (g >= R) return;
    const int k = g;
    const int64_t rr = R * row + k;
    const double* wp = W + rr * ldw + 4 * q;
    float out[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float h = sh[c], l = sl[c];
        if (R == 3) {
            h = k == 0 ? sh[c] : (k == 1 ? sh[4 + c] : sh[8 + c]);
            l = k == 0 ? sl[c] : (k == 1 ? sl[4 + c] : sl[8 + c]);
        }
        out[c] = (float)((wp[c] - (double)h) - (double)l);
    }
    reinterpret_cast<float4*>(r + rr * 32)[q] = make_float4(out[0], out[1], out[2], out[3]);
    if (x1) {   // first semi-iteration step on r, as dscale_kernel computes it
        const float d = inv_theta * dinv[row];
        reinterpret_cast<float4*>(x1 + rr * 32)[q] = make_float4(d * out[0], d * out[1], d * out[2], d * out[3]);
    }
}

int launch_split(int64_t rows, int b, const double* X, int64_t ldx, float* Xh, float* Xl, cudaStream_t s) {
    if (rows * b == 0) return NM_OK;
    split_kernel<<<grid_for(rows * b), kThreads, 0, s>>>(rows, b, X, ldx, Xh, Xl);
    count_launch();
    NM_CUDA(cudaGetLastError());
    return NM_OK;
}

int launch_bsr33_df(const Bsr33DfArgs& a, cudaStream_t s) {
    if (a.b < 1 || a.b > 64) return fail(NM_EINVAL, "block width must be in 1..64");
    if (a.vec && a.b == 32 && (((uintptr_t)a.Xh | (uintptr_t)a.Xl) & 15) == 0) {
        const int nt = a.nt;
        const int64_t grid = (a.nrows + nt / 32 - 1) / (nt / 32);
        if (grid == 0) return NM_OK;
        switch (nt) {
            case 32: bsr33_df_v4_kernel<32><<<(unsigned)grid, 32, 0, s>>>(a); break;
            case 64: bsr33_df_v4_kernel<64><<<(unsigned)grid, 64, 0, s>>>(a); break;
            case 128: bsr33_df_v4_kernel<128><<<(unsigned)grid, 128, 0, s>>>(a); break;
            default: bsr33_df_v4_kernel<256><<<(unsigned)grid, 256, 0, s>>>(a); break;
        }
        count_launch();
        NM_CUDA(cudaGetLastError());
        return NM_OK;
    }
    const int shift = tpr_shift_for(a.b);
    const int cpt = (a.b + (1 << shift) - 1) >> shift;
    const int64_t grid = (a.nrows + (kThreads >> shift) - 1) / (kThreads >> shift);
    if (grid == 0) return NM_OK;
    if (cpt == 1)
        bsr33_df_kernel<1><<<(unsigned)grid, kThreads, 0, s>>>(a, shift);
    else
        bsr33_df_kernel<2><<<(unsigned)grid, kThreads, 0, s>>>(a, shift);
    count_launch();
    NM_CUDA(cudaGetLastError());
    return NM_OK;
}

int launch_resid_df(int R, int64_t nodes, const int* rowptr, const int* col, const float* vh, const float* vl,
                    const double* W, int64_t ldw, const float* x32, float* r32, int b, cudaStream_t s, int vec,
                    int nt, const float* dinv, float inv_theta, float* x1) {
    if (b < 1 || b > 64) return fail(NM_EINVAL, "block width must be in 1..64");
    if (vec && b == 32 && (((uintptr_t)x32 | (uintptr_t)r32 | (uintptr_t)x1) & 15) == 0) {
        if (nt != 32 && nt != 64 && nt != 128) nt = 256;
        const int64_t grid = (nodes + nt / 32 - 1) / (nt / 32);
        if (grid == 0) return NM_OK;
#define NM_RESID_V4(RR, NN) \
    resid_df_v4_kernel<RR, NN><<<(unsigned)grid, NN, 0, s>>>(nodes, rowptr, col, vh, vl, W, ldw, x32, r32, dinv, \
                                                            inv_theta, x1)
        if (R == 3) {
            switch (nt) {
                case 32: NM_RESID_V4(3, 32); break;
                case 64: NM_RESID_V4(3, 64); break;
                case 128: NM_RESID_V4(3, 128); break;
                default: NM_RESID_V4(3, 256); break;
            }
        } else {
            switch (nt) {
                case 32: NM_RESID_V4(1, 32); break;
                case 64: NM_RESID_V4(1, 64); break;
                case 128: NM_RESID_V4(1, 128); break;
                default: NM_RESID_V4(1, 256); break;
            }
        }
#undef NM_RESID_V4
        count_launch();
        NM_CUDA(cudaGetLastError());
        return NM_OK;
    }
    const int shift = tpr_shift_for(b);
    const int cpt = (b + (1 << shift) - 1) >> shift;
    const int64_t grid = (nodes + (kThreads >> shift) - 1) / (kThreads >> shift);
    if (grid == 0) return NM_OK;
    if (R == 3 && cpt == 1)
        resid_df_kernel<3, 1><<<(unsigned)grid, kThreads, 0, s>>>(nodes, rowptr, col, vh, vl, W, ldw, x32, r32, b, shift);
    else if (R == 3)
        resid_df_kernel<3, 2><<<(unsigned)grid, kThreads, 0, s>>>(nodes, rowptr, col, vh, vl, W, ldw, x32, r32, b, shift);
    else if (cpt == 1)
        resid_df_kernel<1, 1><<<(unsigned)grid, kThreads, 0, s>>>(nodes, rowptr, col, vh, vl, W, ldw, x32, r32, b, shift);
    else
        resid_df_kernel<1, 2><<<(unsigned)grid, kThreads, 0, s>>>(nodes, rowptr, col, vh, vl, W, ldw, x32, r32, b, shift);
    count_launch();
    NM_CUDA(cudaGetLastError());
    if (x1) return launch_dscale<float>(R, nodes, b, inv_theta, dinv, r32, b, x1, b, s);
    return NM_OK;
}

// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two
// 32x32->64 multiplies with the published multipliers and Weyl key bumps.
__device__ inline void philox_round(uint32_t c[4], uint32_t k[2]) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k[0];
    const uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

__global__ void philox_normal_kernel(int64_t count, uint64_t seed, double* out) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; 2 * t < count;
         t += (int64_t)gridDim.x * blockDim.x) {
        uint32_t c[4] = {(uint32_t)t, (uint32_t)(t >> 32), 0u, 0u};
        uint32_t k[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
        for (int r = 0; r < 10; ++r) {
            philox_round(c, k);
            k[0] += 0x9E3779B9u;
            k[1] += 0xBB67AE85u;
        }
        // two uniforms in (0, 1) with 53-bit resolution, then Box-Muller
        const double u1 = ((double)(((uint64_t)c[0] << 21) ^ c[1]) + 0.5) * 0x1p-53;
        const double u2 = ((double)(((uint64_t)c[2] << 21) ^ c[3]) + 0.5) * 0x1p-53;
        const double r = sqrt(-2.0 * log(u1));
        const double th = 6.283185307179586 * u2;
        out[2 * t] = r * cos(th);
        if (2 * t + 1 < count) out[2 * t + 1] = r * sin(th);
    }
}

int launch_philox_normal(int64_t count, uint64_t seed, double* out, cudaStream_t s) {
    if (count == 0) return NM_OK;
    philox_normal_kernel<<<grid_for((count + 1) / 2), kThreads, 0, s>>>(count, seed, out);
    count_launch();
    NM_CUDA(cudaGetLastError());
    return NM_OK;
}

template int launch_kron<double>(int, int, const KronArgs<double>&, cudaStream_t);
template int launch_kron<float>(int, int, const KronArgs<float>&, cudaStream_t);
template int launch_bsr33<double>(const Bsr33Args<double>&, cudaStream_t);
template int launch_bsr33<float>(const Bsr33Args<float>&, cudaStream_t);
template int launch_bsr13<double>(const Bsr13Args<double>&, cudaStream_t);
template int launch_bsr13<float>(const Bsr13Args<float>&, cudaStream_t);
template int launch_dscale<double>(int, int64_t, int, double, const double*, const double*, int64_t, double*, int64_t, cudaStream_t);
template int launch_dscale<float>(int, int64_t, int, float, const float*, const float*, int64_t, float*, int64_t, cudaStream_t);
template int launch_scale_copy<double>(int64_t, int, double, const double*, int64_t, double*, int64_t, cudaStream_t);
template int launch_scale_copy<float>(int64_t, int, float, const float*, int64_t, float*, int64_t, cudaStream_t);
template int launch_convert<double, float>(int64_t, int, const double*, int64_t, float*, int64_t, cudaStream_t);
template int launch_convert<float, double>(int64_t, int, const float*, int64_t, double*, int64_t, cudaStream_t);

}  // namespace nm
