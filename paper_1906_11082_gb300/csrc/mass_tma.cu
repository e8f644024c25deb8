// Shared-memory staged float mass step for sm_103a.
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
// per SM walks its tiles with a three-stage pipeline:
//  - warps 0..2 (producers) wait until a stage is free, then fill it: the
//    tile's distinct neighbour records by 16-byte cp.async copies (threads
//    cover consecutive bytes of a record; each thread's copies arrive on
//    the stage's mbarrier when they land), and by cp.async.bulk (complete_tx
//    on the same mbarrier) the tile's rows of w and x_{k-1} and 16-byte
//    windows of its matrix values, local column indices, row pointers,
//    inverse diagonal and own-node positions. The records go through
//    cp.async rather than one bulk copy each: at 384 bytes a copy, the
//    bulk-copy unit's per-copy cost made the step 2.3x slower than the
//    cached gathers it replaces;
//  - warps 3..10 (consumers) wait for the stage; warp c takes rows
//    r0 + 4c .. r0 + 4c + 3, one per group of eight lanes: lane q of a
//    group walks its row's entries, reads each neighbour record's columns
//    4q..4q+3 of the three components from shared memory (16-byte reads),
//    applies the update to them and stores x_{k+1}; no partial sums cross
//    lanes. w and x_{k-1} of the next tile's rows are loaded into
//    registers while the current tile is computed. Then the warp releases
//    the stage.
// Each neighbour record thus crosses L2 -> SM about 6 times per row
// instead of 27, and every HBM / L2 latency is hidden behind the other
// stages.
//
// Every wait is bounded (about one second of clock cycles): on time-out
// the waiting warp sets the error flag, the producers wait for their own
// copies still in flight, and the CTA returns; the host reads the flag
// with tma_status.
#include <cstdio>
#include <vector>

#include "kernels.h"
#include "nm_internal.h"

namespace nm {

namespace {

constexpr int kProducers = 3;                    // producer warps
constexpr int kConsumers = 8;                    // consumer warps
constexpr int kThreadsTma = 32 * (kProducers + kConsumers);
constexpr int kStages = 3;
constexpr int kRec = 96;                         // floats per node record (3 x 32)
constexpr int kRecBytes = kRec * 4;              // 384
constexpr int kChunks = kRecBytes / 16;          // 16-byte pieces of a record (24)
// stage layout (bytes; every piece starts on a 16-byte boundary)
constexpr int kOffRec = 0;
constexpr int kOffVal = kOffRec + kTmaDcap * kRecBytes;
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
constexpr int kMetaInts = kTmaDcap + 16;                 // node-id window of one tile
constexpr int kSmemBytes = kStages * kStageBytes + 2 * kMetaInts * 4 + 128;   // + node ids, mbarriers
static_assert(kOffVal % 16 == 0 && kOffLcol % 16 == 0 && kOffRowp % 16 == 0 && kOffDinv % 16 == 0 &&
                  kOffDiag % 16 == 0,
              "stage pieces must be 16-byte aligned");
static_assert(kSmemBytes <= 227 * 1024, "stages exceed the shared memory of a CTA");
static_assert(kTmaRows == 4 * kConsumers, "a consumer warp takes four rows, one per group of eight lanes");
static_assert((32 * kProducers) % kChunks == 0, "producer threads must cover whole records");

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

// One try: the thread may sleep in it until the phase completes or a
// 20-microsecond hint runs out, so waiting warps take few issue slots.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(20000u)
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

// 16-byte asynchronous copy global -> shared (L2 only).
__device__ __forceinline__ void cp16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// Arrive on `bar` once every cp.async this thread issued so far has landed
// (counts as one of the barrier's expected arrivals).
__device__ __forceinline__ void cp_async_arrive(uint64_t* bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void producers_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(32 * kProducers) : "memory");
}

// Barrier of the producer threads that also ANDs a flag over them, so that
// every producer takes the same branch after its bounded waits.
__device__ __forceinline__ bool producers_all(bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "n"(32 * kProducers)
        : "memory");
    return r != 0;
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

// Streamed own-row operands (w, x_{k-1}) of a lane's row of a tile:
// columns 4q..4q+3 of each component.
struct RowOps {
    float4 w[3], xp[3];
};

__device__ __forceinline__ void load_rowops(const KronArgs<float>& a, int row, bool valid, int q, bool has_xp,
                                            RowOps& o) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int64_t idx = (3 * (int64_t)row + k) * 8 + q;   // float4 index
        o.w[k] = valid ? __ldcs(reinterpret_cast<const float4*>(a.W) + idx) : make_float4(0.f, 0.f, 0.f, 0.f);
        o.xp[k] = (valid && has_xp) ? __ldcs(reinterpret_cast<const float4*>(a.Xp) + idx)
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

__global__ void __launch_bounds__(kThreadsTma, 1) kron_tma_kernel(const KronArgs<float> a) {
    extern __shared__ __align__(128) unsigned char smem[];
    int* meta = reinterpret_cast<int*>(smem + kStages * kStageBytes);          // 2 x kMetaInts node ids
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kStages * kStageBytes + 2 * kMetaInts * 4);
    uint64_t* empty = full + kStages;
    uint64_t* mbar = empty + kStages;                                           // 2 node-id slots
    const TmaTiles& T = a.tma;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            // every producer thread's cp.async arrival, plus the bulk copies' expect_tx arrival
            mbar_init(full + s, 32 * kProducers + 1);
            mbar_init(empty + s, kConsumers);
        }
        mbar_init(mbar, 1);
        mbar_init(mbar + 1, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool has_xp = a.Xp != nullptr;
    if (warp < kProducers) {
        // ------------------------------------------------------------ producers
        // Tile metadata runs one tile ahead: the descriptor and row-pointer
        // bounds of tile i + 1 are in registers, and its node-id list is on
        // its way into the other node-id slot, while tile i is copied.
        const int pt = threadIdx.x;                       // 0 .. 32 kProducers - 1
        const int off = pt % kChunks, rsub = pt / kChunks;
        constexpr int kRecStep = 32 * kProducers / kChunks;   // records per producer round (4)
        const int G = gridDim.x;
        auto meta_copy = [&](int slot, int4 dd) {
            const Window wu = window(dd.z, dd.z + dd.w, 4);
            mbar_arrive_expect_tx(mbar + slot, wu.bytes);
            bulk_g2s(meta + slot * kMetaInts, T.ucol + wu.base, wu.bytes, mbar + slot);
        };
        int4 dn = make_int4(0, 0, 0, 0);
        int en0 = 0, en1 = 0;
        bool meta_pending = false;   // a node-id copy is in flight (for the error path)
        if ((int)blockIdx.x < T.ntiles) {
            dn = __ldg(T.desc + blockIdx.x);
            en0 = __ldg(T.rowptr + dn.x);
            en1 = __ldg(T.rowptr + dn.y);
            if (pt == 0) meta_copy(0, dn);
            meta_pending = true;
        }
        int i = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < T.ntiles; t += G, ++i) {
            const int s = i % kStages, use = i / kStages, ms = i & 1;
            const int4 d = dn;
            const int e0 = en0, e1 = en1;
            bool next = t + G < T.ntiles;
            if (next) {
                dn = __ldg(T.desc + t + G);
                en0 = __ldg(T.rowptr + dn.x);
                en1 = __ldg(T.rowptr + dn.y);
                if (pt == 0) {
                    // the other slot was last read in the previous iteration, before its closing barrier
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    meta_copy(ms ^ 1, dn);
                }
            }
            bool w_ok = use == 0 || mbar_wait(empty + s, (use - 1) & 1);
            w_ok = mbar_wait(mbar + ms, (i >> 1) & 1) && w_ok;
            meta_pending = next;
            if (!producers_all(w_ok)) {
                ok = false;
                break;
            }
            const int r0 = d.x, r1 = d.y, u0 = d.z, nu = d.w;
            const int* nodes = meta + ms * kMetaInts + (u0 & 3);
            unsigned char* st = smem + s * kStageBytes;
            if (pt == 0) {
                const Window wv = window(e0, e1, 4), wl = window(e0, e1, 2), wr = window(r0, r1 + 1, 4),
                             wd = window(r0, r1, 4), wg = window(r0, r1, 2);
                mbar_arrive_expect_tx(full + s, wv.bytes + wl.bytes + wr.bytes + wd.bytes + wg.bytes);
                bulk_g2s(st + kOffVal, T.vals + wv.base, wv.bytes, full + s);
                bulk_g2s(st + kOffLcol, T.lcol + wl.base, wl.bytes, full + s);
                bulk_g2s(st + kOffRowp, T.rowptr + wr.base, wr.bytes, full + s);
                bulk_g2s(st + kOffDinv, T.dinv + wd.base, wd.bytes, full + s);
                bulk_g2s(st + kOffDiag, T.ldiag + wg.base, wg.bytes, full + s);
            }
            // neighbour records: thread (rsub, off) copies piece `off` of
            // records rsub, rsub + 4, ...; 24 consecutive threads cover one
            // record's 384 contiguous bytes
            unsigned char* rec = st + kOffRec + off * 16;
            const float* src = a.X + off * 4;
            int r = rsub;
            for (; r + 3 * kRecStep < nu; r += 4 * kRecStep) {
                const int n0 = nodes[r], n1 = nodes[r + kRecStep], n2 = nodes[r + 2 * kRecStep],
                          n3 = nodes[r + 3 * kRecStep];
                cp16(rec + r * kRecBytes, src + (int64_t)n0 * kRec);
                cp16(rec + (r + kRecStep) * kRecBytes, src + (int64_t)n1 * kRec);
                cp16(rec + (r + 2 * kRecStep) * kRecBytes, src + (int64_t)n2 * kRec);
                cp16(rec + (r + 3 * kRecStep) * kRecBytes, src + (int64_t)n3 * kRec);
            }
            for (; r < nu; r += kRecStep) cp16(rec + r * kRecBytes, src + (int64_t)nodes[r] * kRec);
            cp_async_arrive(full + s);
            producers_sync();   // this node-id slot is refilled two tiles on
        }
        if (!ok) {
            if (pt == 0) atomicExch(T.err, 1);
            // let the copies already issued land before the CTA's shared memory goes away
            asm volatile("cp.async.wait_all;" ::: "memory");
            for (int j = i - 1; j >= 0 && j >= i - kStages; --j) mbar_wait(full + (j % kStages), (j / kStages) & 1);
            if (meta_pending) mbar_wait(mbar + ((i + 1) & 1), ((i + 1) >> 1) & 1);
        }
        return;
    }
    // ---------------------------------------------------------------- consumers
    // Consumer warp c takes rows r0 + 4c .. r0 + 4c + 3 of each tile, one
    // per group of eight lanes; lane q of a group owns columns 4q..4q+3 of
    // the three components of its row, so no partial sums cross lanes.
    const int c = warp - kProducers;
    const int g = lane >> 3, q = lane & 7;
    const int lr = 4 * c + g;   // the lane's row within a tile
    const float inv_theta = a.inv_theta, om = a.om;
    // the streamed own-row operands are loaded one tile ahead, into registers
    RowOps cur, nxt;
    int4 dn = make_int4(0, 0, 0, 0);
    if ((int)blockIdx.x < T.ntiles) {
        dn = __ldg(T.desc + blockIdx.x);
        load_rowops(a, dn.x + lr, dn.x + lr < dn.y, q, has_xp, nxt);
    }
    int i = 0;
    for (int t = blockIdx.x; t < T.ntiles; t += gridDim.x, ++i) {
        const int s = i % kStages, use = i / kStages;
        const int4 d = dn;
        cur = nxt;
        if (t + (int)gridDim.x < T.ntiles) {
            dn = __ldg(T.desc + t + gridDim.x);
            load_rowops(a, dn.x + lr, dn.x + lr < dn.y, q, has_xp, nxt);
        }
        if (!mbar_wait(full + s, use & 1)) {
            if (lane == 0) atomicExch(T.err, 2);
            return;
        }
        const unsigned char* st = smem + s * kStageBytes;
        const float4* rec = reinterpret_cast<const float4*>(st + kOffRec) + q;
        const float* vs = reinterpret_cast<const float*>(st + kOffVal);
        const uint16_t* ls = reinterpret_cast<const uint16_t*>(st + kOffLcol);
        const int* rps = reinterpret_cast<const int*>(st + kOffRowp);
        const float* dis = reinterpret_cast<const float*>(st + kOffDinv);
        const uint16_t* dgs = reinterpret_cast<const uint16_t*>(st + kOffDiag);
        const int r0 = d.x, r1 = d.y;
        const int row = r0 + lr;
        if (row < r1) {
            const int rb = r0 & ~3, db = r0 & ~7;
            const int e0 = rps[r0 - rb];
            const int vb = e0 & ~3, lb = e0 & ~7;
            const int ea = rps[row - rb], eb = rps[row + 1 - rb];
            float4 acc[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) acc[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            int e = ea;
            for (; e + 1 < eb; e += 2) {
                const float v0 = vs[e - vb], v1 = vs[e + 1 - vb];
                const float4* p0 = rec + ls[e - lb] * (kRec / 4);
                const float4* p1 = rec + ls[e + 1 - lb] * (kRec / 4);
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
                const float4* p0 = rec + ls[e - lb] * (kRec / 4);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float4 x0 = p0[8 * k];
                    acc[k].x += v0 * x0.x;
                    acc[k].y += v0 * x0.y;
                    acc[k].z += v0 * x0.z;
                    acc[k].w += v0 * x0.w;
                }
            }
            const float dd = dis[row - rb] * inv_theta;
            const float4* own = rec + dgs[row - db] * (kRec / 4);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float4 xk = own[8 * k], w = cur.w[k], xp = cur.xp[k];
                float4 xn;
                xn.x = xp.x + om * (xk.x - xp.x + dd * (w.x - acc[k].x));
                xn.y = xp.y + om * (xk.y - xp.y + dd * (w.y - acc[k].y));
                xn.z = xp.z + om * (xk.z - xp.z + dd * (w.z - acc[k].z));
                xn.w = xp.w + om * (xk.w - xp.w + dd * (w.w - acc[k].w));
                __stcs(reinterpret_cast<float4*>(a.Xn) + (3 * (int64_t)row + k) * 8 + q, xn);
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
    ucol.resize(ucol.size() + 16, 0);   // 16-byte windows never leave the allocation
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
