// Bulk-copy staged float mass step for sm_103a.
//
// One Jacobi-Chebyshev semi-iteration step of the mass solve (the inner
// M^{-1} "by matrix-vector products" of the filter, Sec. 6.2),
//
//     x_{k+1} = x_{k-1} + om (x_k - x_{k-1} + D^{-1} (w - (M_rho (x) I_3) x_k) / theta),
//
// on a block of 32 float columns (row-major, ld 32, so a node's three
// component rows are one contiguous 384-byte record).
//
// The gather of neighbour records dominates this step: each row reads ~27
// records of 384 B, ten times the bytes the step must move. Rows are in a
// Morton order, so consecutive rows share most neighbours; the rows are
// cut into tiles of at most 32 rows whose union of neighbours holds at
// most 192 nodes (built on the host, once per matrix). A persistent CTA
// per SM walks its tiles with a two-stage pipeline:
//  - warp 0 (producer) waits until a stage is free, then copies into it
//    with cp.async.bulk (completion on the stage's mbarrier): every
//    distinct neighbour record of the tile, the tile's rows of w and
//    x_{k-1}, and 16-byte windows of the tile's matrix values, local column
//    indices, row pointers, inverse diagonal and own-node positions;
//  - warps 1..8 (consumers) wait for the stage, each takes rows r0 + c,
//    r0 + c + 8, ...: four groups of eight lanes take the row's entries
//    g, g + 4, ... and read the neighbour's record from shared memory
//    (lane q: columns 4q..4q+3 of each component, 16-byte reads), the
//    partial sums are combined by shuffles and lane c applies the update
//    to column c and stores x_{k+1}; then the warp releases the stage.
// Each neighbour record thus crosses L2 -> SM about 6 times per row
// instead of 27, and every HBM / L2 latency is hidden behind the other
// stage.
//
// Every wait is bounded (about one second of clock cycles): on time-out
// the waiting warp sets the error flag, the producer waits (bounded) for
// its own copies still in flight, and the CTA returns; the host reads the
// flag with tma_status.
#include <cstdio>
#include <vector>

#include "kernels.h"
#include "nm_internal.h"

namespace nm {

namespace {

constexpr int kConsumers = 8;
constexpr int kThreadsTma = 32 * (kConsumers + 1);
constexpr int kStages = 2;
constexpr int kRec = 96;                         // floats per node record (3 x 32)
constexpr int kRecBytes = kRec * 4;              // 384
// stage layout (bytes; every piece starts on a 16-byte boundary)
constexpr int kOffRec = 0;
constexpr int kOffW = kOffRec + kTmaDcap * kRecBytes;
constexpr int kOffXp = kOffW + kTmaRows * kRecBytes;
constexpr int kOffVal = kOffXp + kTmaRows * kRecBytes;
constexpr int kValSlots = kTmaEcap + 16;
constexpr int kOffLcol = kOffVal + kValSlots * 4;
constexpr int kLcolSlots = kTmaEcap + 16;
constexpr int kOffRowp = kOffLcol + kLcolSlots * 2;
constexpr int kRowpSlots = kTmaRows + 8;
constexpr int kOffDinv = kOffRowp + kRowpSlots * 4;
constexpr int kDinvSlots = kTmaRows + 8;
constexpr int kOffDiag = kOffDinv + kDinvSlots * 4;
constexpr int kDiagSlots = kTmaRows + 16;
constexpr int kStageBytes = ((kOffDiag + kDiagSlots * 2) + 127) / 128 * 128;
constexpr int kSmemBytes = kStages * kStageBytes + 128;   // + the mbarriers
static_assert(kOffW % 16 == 0 && kOffXp % 16 == 0 && kOffVal % 16 == 0 && kOffLcol % 16 == 0 &&
                  kOffRowp % 16 == 0 && kOffDinv % 16 == 0 && kOffDiag % 16 == 0,
              "stage pieces must be 16-byte aligned");
static_assert(kSmemBytes <= 227 * 1024, "stages exceed the shared memory of a CTA");

constexpr long long kWaitCycles = 2000000000LL;   // ~1 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity; false on time-out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitCycles) return false;
    return true;
}

// 1-D bulk copy global -> shared of `bytes` (multiple of 16, both
// addresses 16-byte aligned), completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

struct Window {
    int base, bytes;
};

// 16-byte window [lo & ~m, (hi + m) & ~m) of elements of size es (m = 16/es - 1).
__device__ __forceinline__ Window window(int lo, int hi, int es) {
    const int m = 16 / es - 1;
    const int b = lo & ~m;
    const int e = (hi + m) & ~m;
    return {b, (e - b) * es};
}

__global__ void __launch_bounds__(kThreadsTma, 1) kron_tma_kernel(const KronArgs<float> a) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes);
    uint64_t* empty = full + kStages;
    const TmaTiles& T = a.tma;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, kConsumers);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool has_xp = a.Xp != nullptr;
    if (warp == 0) {
        // ------------------------------------------------------------ producer
        int i = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < T.ntiles; t += gridDim.x, ++i) {
            const int s = i & 1, use = i >> 1;
            if (use > 0 && !mbar_wait(empty + s, (use - 1) & 1)) {
                ok = false;
                break;
            }
            const int4 d = __ldg(T.desc + t);
            const int r0 = d.x, r1 = d.y, u0 = d.z, nu = d.w;
            const int e0 = __ldg(T.rowptr + r0), e1 = __ldg(T.rowptr + r1);
            const Window wv = window(e0, e1, 4), wl = window(e0, e1, 2), wr = window(r0, r1 + 1, 4),
                         wd = window(r0, r1, 4), wg = window(r0, r1, 2);
            const unsigned rows_bytes = (unsigned)(r1 - r0) * kRecBytes;
            const unsigned total = (unsigned)nu * kRecBytes + rows_bytes * (has_xp ? 2u : 1u) + wv.bytes + wl.bytes +
                                   wr.bytes + wd.bytes + wg.bytes;
            unsigned char* st = smem + s * kStageBytes;
            if (lane == 0) mbar_arrive_expect_tx(full + s, total);
            __syncwarp();
            switch (lane) {
                case 0: bulk_g2s(st + kOffVal, T.vals + wv.base, wv.bytes, full + s); break;
                case 1: bulk_g2s(st + kOffLcol, T.lcol + wl.base, wl.bytes, full + s); break;
                case 2: bulk_g2s(st + kOffRowp, T.rowptr + wr.base, wr.bytes, full + s); break;
                case 3: bulk_g2s(st + kOffDinv, T.dinv + wd.base, wd.bytes, full + s); break;
                case 4: bulk_g2s(st + kOffDiag, T.ldiag + wg.base, wg.bytes, full + s); break;
                case 5: bulk_g2s(st + kOffW, a.W + (int64_t)r0 * kRec, rows_bytes, full + s); break;
                case 6:
                    if (has_xp) bulk_g2s(st + kOffXp, a.Xp + (int64_t)r0 * kRec, rows_bytes, full + s);
                    break;
                default: break;
            }
            // neighbour records: node ids first (independent loads), then the copies
            int node[kTmaDcap / 32];
#pragma unroll
            for (int k = 0; k < kTmaDcap / 32; ++k) {
                const int q = lane + 32 * k;
                node[k] = q < nu ? __ldg(T.ucol + u0 + q) : 0;
            }
#pragma unroll
            for (int k = 0; k < kTmaDcap / 32; ++k) {
                const int q = lane + 32 * k;
                if (q < nu) bulk_g2s(st + kOffRec + q * kRecBytes, a.X + (int64_t)node[k] * kRec, kRecBytes, full + s);
            }
        }
        if (!ok) {
            if (lane == 0) atomicExch(T.err, 1);
            // let the copies already issued land before the CTA's shared memory goes away
            const int issued = i;
            for (int j = issued - 1; j >= 0 && j >= issued - kStages; --j) mbar_wait(full + (j & 1), (j >> 1) & 1);
        }
        return;
    }
    // ---------------------------------------------------------------- consumers
    const int c = warp - 1;
    const int g = lane >> 3, q = lane & 7;
    const float inv_theta = a.inv_theta, om = a.om;
    int i = 0;
    for (int t = blockIdx.x; t < T.ntiles; t += gridDim.x, ++i) {
        const int s = i & 1, use = i >> 1;
        const int4 d = __ldg(T.desc + t);
        if (!mbar_wait(full + s, use & 1)) {
            if (lane == 0) atomicExch(T.err, 2);
            return;
        }
        const unsigned char* st = smem + s * kStageBytes;
        const float* rec = reinterpret_cast<const float*>(st + kOffRec);
        const float* ws = reinterpret_cast<const float*>(st + kOffW);
        const float* xps = reinterpret_cast<const float*>(st + kOffXp);
        const float* vs = reinterpret_cast<const float*>(st + kOffVal);
        const uint16_t* ls = reinterpret_cast<const uint16_t*>(st + kOffLcol);
        const int* rps = reinterpret_cast<const int*>(st + kOffRowp);
        const float* dis = reinterpret_cast<const float*>(st + kOffDinv);
        const uint16_t* dgs = reinterpret_cast<const uint16_t*>(st + kOffDiag);
        const int r0 = d.x, r1 = d.y;
        const int rb = r0 & ~3, db = r0 & ~7;
        const int e0 = rps[r0 - rb];
        const int vb = e0 & ~3, lb = e0 & ~7;
        for (int row = r0 + c; row < r1; row += kConsumers) {
            const int ea = rps[row - rb], eb = rps[row + 1 - rb];
            float4 acc[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) acc[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            int e = ea + g;
            for (; e + 4 < eb; e += 8) {
                const float v0 = vs[e - vb], v1 = vs[e + 4 - vb];
                const float4* p0 = reinterpret_cast<const float4*>(rec + ls[e - lb] * kRec) + q;
                const float4* p1 = reinterpret_cast<const float4*>(rec + ls[e + 4 - lb] * kRec) + q;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float4 x0 = p0[8 * k], x1 = p1[8 * k];
                    acc[k].x += v0 * x0.x + v1 * x1.x;
                    acc[k].y += v0 * x0.y + v1 * x1.y;
                    acc[k].z += v0 * x0.z + v1 * x1.z;
                    acc[k].w += v0 * x0.w + v1 * x1.w;
                }
            }
            if (e < eb) {
                const float v0 = vs[e - vb];
                const float4* p0 = reinterpret_cast<const float4*>(rec + ls[e - lb] * kRec) + q;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float4 x0 = p0[8 * k];
                    acc[k].x += v0 * x0.x;
                    acc[k].y += v0 * x0.y;
                    acc[k].z += v0 * x0.z;
                    acc[k].w += v0 * x0.w;
                }
            }
            // lanes q, q + 8, q + 16, q + 24 hold partial sums of the same columns
#pragma unroll
            for (int k = 0; k < 3; ++k) {
#pragma unroll
                for (int m = 8; m <= 16; m *= 2) {
                    acc[k].x += __shfl_xor_sync(0xffffffffu, acc[k].x, m);
                    acc[k].y += __shfl_xor_sync(0xffffffffu, acc[k].y, m);
                    acc[k].z += __shfl_xor_sync(0xffffffffu, acc[k].z, m);
                    acc[k].w += __shfl_xor_sync(0xffffffffu, acc[k].w, m);
                }
            }
            // column lane lives in element (lane & 3) of lane lane >> 2
            const int src = lane >> 2, sel = lane & 3;
            const int lr = row - r0;
            const float dd = dis[row - rb] * inv_theta;
            const float* own = rec + dgs[row - db] * kRec;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float t0 = __shfl_sync(0xffffffffu, acc[k].x, src);
                const float t1 = __shfl_sync(0xffffffffu, acc[k].y, src);
                const float t2 = __shfl_sync(0xffffffffu, acc[k].z, src);
                const float t3 = __shfl_sync(0xffffffffu, acc[k].w, src);
                const float ax = sel == 0 ? t0 : (sel == 1 ? t1 : (sel == 2 ? t2 : t3));
                const float xk = own[k * 32 + lane];
                const float w = ws[lr * kRec + k * 32 + lane];
                const float xp = has_xp ? xps[lr * kRec + k * 32 + lane] : 0.f;
                const float xn = xp + om * (xk - xp + dd * (w - ax));
                __stcs(a.Xn + (3 * (int64_t)row + k) * 32 + lane, xn);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(empty + s);
    }
}

int g_sm_count = 0;

}  // namespace

int launch_kron_tma(const KronArgs<float>& a, cudaStream_t s) {
    if (a.tma.ntiles <= 0) return fail(NM_EINVAL, "staged mass step without tiles");
    if (a.b != 32 || a.ldx != 32 || a.ldw != 32 || a.ldn != 32 || (a.Xp && a.ldp != 32))
        return fail(NM_EINVAL, "staged mass step needs 32 columns with ld 32");
    if (((uintptr_t)a.X | (uintptr_t)a.W | (uintptr_t)(a.Xp ? a.Xp : a.X)) & 15)
        return fail(NM_EINVAL, "staged mass step needs 16-byte aligned blocks");
    static bool attr = false;
    if (!attr) {
        NM_CUDA(cudaFuncSetAttribute(kron_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
        int dev = 0;
        NM_CUDA(cudaGetDevice(&dev));
        NM_CUDA(cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev));
        attr = true;
    }
    const int grid = std::min(a.tma.ntiles, std::max(g_sm_count, 1));
    kron_tma_kernel<<<grid, kThreadsTma, kSmemBytes, s>>>(a);
    count_launch();
    NM_CUDA(cudaGetLastError());
    return NM_OK;
}

int tma_status(int* err_dev, cudaStream_t s) {
    if (!err_dev) return NM_OK;
    int h = 0;
    NM_CUDA(cudaMemcpyAsync(&h, err_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
    NM_CUDA(cudaStreamSynchronize(s));
    if (h != 0) {
        NM_CUDA(cudaMemsetAsync(err_dev, 0, sizeof(int), s));
        return fail(NM_ETIMEOUT, std::string("a staged mass-step wait ran out (") +
                                     (h == 1 ? "producer" : "consumer") + ")");
    }
    return NM_OK;
}

// Tiles of the scalar CSR A for the staged kernel: greedy over the rows in
// their (Morton) order, closing a tile before it would exceed kTmaRows
// rows, kTmaDcap distinct neighbours or kTmaEcap entries. A row that alone
// exceeds a cap makes the matrix ineligible (state -1).
int build_tma_tiles(DevCSR& A, cudaStream_t s) {
    if (A.tma_state != 0) return NM_OK;
    A.tma_state = -1;
    const int64_t n = A.nrows;
    if (n <= 0 || A.h_rowptr.size() != (size_t)n + 1 || !A.val32.p || !A.dinv32.p) return NM_OK;
    const std::vector<int32_t>& rp = A.h_rowptr;
    const std::vector<int32_t>& ci = A.h_col;
    std::vector<int> mark(n, -1), pos(n, 0);
    std::vector<int4> desc;
    std::vector<int32_t> ucol;
    std::vector<uint16_t> lcol(A.nnz + 16, 0), ldiag(n + 16, 0);
    int64_t r = 0;
    int t = 0;
    while (r < n) {
        const int64_t r0 = r;
        const int u0 = (int)ucol.size();
        int nu = 0;
        while (r < n && r - r0 < kTmaRows) {
            int add = 0;
            for (int e = rp[r]; e < rp[r + 1]; ++e)
                if (mark[ci[e]] != t) ++add;
            if (nu + add > kTmaDcap || rp[r + 1] - rp[r0] > kTmaEcap) break;
            for (int e = rp[r]; e < rp[r + 1]; ++e) {
                const int j = ci[e];
                if (mark[j] != t) {
                    mark[j] = t;
                    pos[j] = nu++;
                    ucol.push_back(j);
                }
                lcol[e] = (uint16_t)pos[j];
            }
            if (mark[r] != t) return NM_OK;   // no diagonal entry: not a mass matrix pattern
            ldiag[r] = (uint16_t)pos[r];
            ++r;
        }
        if (r == r0) return NM_OK;   // one row beyond the caps
        desc.push_back(make_int4((int)r0, (int)r, u0, nu));
        ++t;
    }
    A.tma_desc.release();
    NM_TRY(A.tma_desc.alloc(desc.size() * sizeof(int4)));
    NM_TRY(A.tma_ucol.alloc(ucol.size() * sizeof(int32_t)));
    NM_TRY(A.tma_lcol.alloc(lcol.size() * sizeof(uint16_t)));
    NM_TRY(A.tma_ldiag.alloc(ldiag.size() * sizeof(uint16_t)));
    NM_TRY(A.tma_vals.alloc((A.nnz + 16) * sizeof(float)));
    NM_TRY(A.tma_rowptr.alloc((n + 1 + 16) * sizeof(int32_t)));
    NM_TRY(A.tma_dinv.alloc((n + 16) * sizeof(float)));
    NM_TRY(A.tma_err.alloc(sizeof(int)));
    NM_CUDA(cudaMemcpyAsync(A.tma_desc.p, desc.data(), desc.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
    NM_CUDA(cudaMemcpyAsync(A.tma_ucol.p, ucol.data(), ucol.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    NM_CUDA(cudaMemcpyAsync(A.tma_lcol.p, lcol.data(), lcol.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, s));
    NM_CUDA(cudaMemcpyAsync(A.tma_ldiag.p, ldiag.data(), ldiag.size() * sizeof(uint16_t), cudaMemcpyHostToDevice,
                            s));
    NM_CUDA(cudaMemsetAsync(A.tma_vals.p, 0, (A.nnz + 16) * sizeof(float), s));
    NM_CUDA(cudaMemcpyAsync(A.tma_vals.p, A.val32.p, A.nnz * sizeof(float), cudaMemcpyDeviceToDevice, s));
    NM_CUDA(cudaMemsetAsync(A.tma_rowptr.p, 0, (n + 1 + 16) * sizeof(int32_t), s));
    NM_CUDA(cudaMemcpyAsync(A.tma_rowptr.p, A.rowptr.p, (n + 1) * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    NM_CUDA(cudaMemsetAsync(A.tma_dinv.p, 0, (n + 16) * sizeof(float), s));
    NM_CUDA(cudaMemcpyAsync(A.tma_dinv.p, A.dinv32.p, n * sizeof(float), cudaMemcpyDeviceToDevice, s));
    NM_CUDA(cudaMemsetAsync(A.tma_err.p, 0, sizeof(int), s));
    NM_CUDA(cudaStreamSynchronize(s));
    TmaTiles& T = A.tma;
    T.ntiles = (int)desc.size();
    T.desc = A.tma_desc.as<int4>();
    T.ucol = A.tma_ucol.as<int>();
    T.lcol = A.tma_lcol.as<uint16_t>();
    T.vals = A.tma_vals.as<float>();
    T.rowptr = A.tma_rowptr.as<int>();
    T.dinv = A.tma_dinv.as<float>();
    T.ldiag = A.tma_ldiag.as<uint16_t>();
    T.err = A.tma_err.as<int>();
    A.tma_state = 1;
    return NM_OK;
}

}  // namespace nm
