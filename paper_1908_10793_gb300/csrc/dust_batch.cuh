// Batched step of many independent instances as one persistent launch
// (instantiated in dust_slab_batch.cu, beside the step kernels of the same
// geometries).
//
// One cooperative launch (every block resident at once) runs all steps of a
// dust_batch_step call for all instances of a batch.  The instances are
// dealt into groups; one step of a group is a chain of phases:
//
//   sort (steps s with s % sort_interval == 0):
//     scan A   chunk sums of the key counts the previous step predicted
//     scan B   exclusive scan of the chunk sums, one item per instance
//     scan C   offsets inside each chunk, copied to the scatter's cursors
//     scatter  (id, source) pairs to their key segments
//     segments id sort inside each key (warp-staged)
//   zero       the deposit, the next sort's key counts; block sort of long
//              segments
//   tiles      the slab step kernel's tile function (gather, push, deposit,
//              next keys, and the sort's gather through the permutation)
//   feedback   the deposit applied to the gas; time advanced
//
// A task is one phase of one step of one group, cut into work items (chunks
// of the per-context kernels' blocks, or tiles).  The host lays the tasks out
// in rounds, group g's phase p of step s in round s * period + g + p, so that
// at any time the groups are in different phases (the sort of one group runs
// beside the tiles of others), and the blocks take work items in that order
// from one counter.  A task waits, bounded in time, until the group's
// previous task has counted all its items done; since items are taken in
// order and every task waits only for earlier ones, the wait always ends
// unless a block stopped.  When a wait runs out the kernel raises
// DUST_FLAG_TIMEOUT in every instance's status words and returns.
//
// Every item runs the same device functions as the per-context kernels, on
// the same buffers, in the same order per instance, so a batch gives the
// grains, gas and deposit of its instances stepped one at a time, bit for
// bit.
#pragma once

#include <algorithm>

#include "dust_slab.cuh"
#include "dust_sort.cuh"

namespace dust {

static_assert(kBatchSegChunk == kSegThreads && kBatchScanChunk == kSlabThreads * kScanItems &&
                  kBatchFbChunk == kSlabThreads,
              "batch chunks are the per-context kernels' blocks");

namespace {

// The sort's buffers of one instance for one sort (the fields the sort's
// device functions read).
struct BatchSort {
    struct {
        const int32_t *id;
        int64_t n;
    } src;
    int32_t *key, *count, *cursor, *pair_id, *pair_src, *big, *tmp_id, *tmp_src;
    int64_t nkeys1;
};

// Thread 0 waits until *count reaches target, at most limit_ns; the result
// is broadcast to the block.  Writes that the counted items made before
// signalling (generic proxy) are then visible to this block's bulk tensor
// copies (async proxy).
__device__ bool wait_count(const int *count, int target, unsigned long long limit_ns)
{
    int ok = 1;
    if (threadIdx.x == 0) {
        const volatile int *c = count;
        if (*c < target) {
            const unsigned long long t0 = global_ns();
            while (*c < target) {
                if (global_ns() - t0 > limit_ns) {
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    ok = __syncthreads_and(ok);
    asm volatile("fence.proxy.async.global;" ::: "memory");
    return ok != 0;
}

// After a work item: every thread's writes, then one count.
__device__ __forceinline__ void signal_done(int *count)
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(count, 1);
    }
}

// Per-instance state of step s: which store is current, which count buffer
// holds the offsets of the last sort (and which the next sort's counts).
struct StepState {
    int cur;   // current store
    int coff;  // count buffer with the offsets the step uses
};

__device__ __forceinline__ StepState state_of(const BatchInst &I, int s, int K)
{
    // sorts before the step (sorts at steps 0, K, 2K, ... of this launch)
    const int sorts_before = s == 0 ? 0 : (s - 1) / K + 1;
    const int sorted = (s % K) == 0;
    StepState st;
    // every sort flips the store (its gather writes the other store) and
    // makes the scanned buffer, count[1] for the first sort, the offsets
    const int flips = sorts_before + sorted;
    st.cur = (I.cur + flips) & 1;
    st.coff = sorts_before + sorted == 0 ? 0 : ((sorts_before + sorted) & 1);
    return st;
}

__device__ __forceinline__ BatchSort sort_of(const BatchInst &I, const StepState &st)
{
    BatchSort a;
    const int src = st.cur ^ 1;  // the store the sort reads (the step gathers from it)
    a.src.id = I.store[src].id;
    a.src.n = I.n;
    a.key = I.key;
    a.count = I.count[st.coff];
    a.cursor = I.cursor;
    a.pair_id = I.pair_id;
    a.pair_src = I.pair_src;
    a.big = I.bigseg;
    a.tmp_id = I.key;
    a.tmp_src = I.store[st.cur].id;
    a.nkeys1 = I.nkeys + 1;
    return a;
}

// One tile of the persistent kernel, out of line: the tile function then
// gets its own register allocation instead of sharing the persistent loop's.
template <int GEOM, int FLAT, int MODE, int TX, int TY, int TZ>
__device__ __noinline__ bool batch_tile(const TiledArgs<float> &TA, int tile, int ntile, unsigned char *smem_raw)
{
    return slab_tile<GEOM, FLAT, MODE, TX, TY, TZ>(TA, tile, ntile, smem_raw, true);
}

}  // namespace

template <int GEOM, int FLAT, int MODE, int TX, int TY, int TZ>
__global__ void __launch_bounds__(kSlabThreads, 2) batch_persistent_kernel(const BatchDev B)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int K = B.sort_interval;
    int32_t *ws = reinterpret_cast<int32_t *>(smem_raw);  // scan: 32 words
    TiledArgs<float> *sTA = reinterpret_cast<TiledArgs<float> *>(smem_raw + B.ta_offset);
    int *s_item = reinterpret_cast<int *>(smem_raw + B.ta_offset + sizeof(TiledArgs<float>));
    bool ok = true;

    // the block takes items in increasing order, so the task of its next item
    // is at or after the task of its last one; and a task the block has
    // already waited for needs no second wait
    int tcache = 0, verified = -1;
    for (;;) {
        __syncthreads();
        if (threadIdx.x < 32) {
            const unsigned FULL = 0xffffffffu;
            const int lane = threadIdx.x;
            int w = lane == 0 ? atomicAdd(B.grab, 1) : 0;
            w = __shfl_sync(FULL, w, 0);
            int t = tcache;
            if (w < B.nitems) {
                // tasks start in increasing order: the tasks after t that
                // start at or before w form a prefix, 32 looked at at once
                for (;;) {
                    const int j = t + 1 + lane;
                    const unsigned m = __ballot_sync(FULL, j < B.ntasks && B.tasks[j].begin <= w);
                    t += __popc(m);
                    if (m != FULL) break;
                }
            }
            if (lane == 0) {
                s_item[0] = w;
                s_item[1] = t;
            }
        }
        __syncthreads();
        const int w = s_item[0];
        if (w >= B.nitems) break;
        const int t = s_item[1];
        tcache = t;
        const BatchTask T = B.tasks[t];
        // the group's previous task must be complete
        if (T.dep >= 0 && T.dep != verified) {
            if (!wait_count(B.done + T.dep, B.tasks[T.dep].items + B.wait_extra, B.wait_ns)) {
                ok = false;
                break;
            }
            verified = T.dep;
        }
        const int s = T.s, p = T.p;
        const bool sorted = (s % K) == 0;
        const bool emit = ((s + 1) % K) == 0;
        // the instance of the group and its item
        const int l = w - T.begin;
        const int *pre = B.gpre + ((size_t)((sorted ? 1 : 0) * BPH_N + p) * B.ngroups + T.g) * (B.gmax + 1);
        int lo = 0, hi = B.gcount[T.g];  // pre[lo] <= l < pre[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (pre[mid] <= l) lo = mid;
            else hi = mid;
        }
        const int i = B.members[T.g * B.gmax + lo];
        const int li = l - pre[lo];
        const BatchInst &I = B.inst[i];
        const StepState st = state_of(I, s, K);
        const int64_t c0 = (int64_t)li * kBatchChunks;  // first chunk of a chunked item

        if (p == BPH_SCANA) {
            const int64_t nscan = (I.nkeys + 2 + kBatchScanChunk - 1) / kBatchScanChunk;
            for (int64_t c = c0; c < min(c0 + kBatchChunks, nscan); ++c) {
                scan_reduce_block(I.count[st.coff], I.nkeys + 2, I.blocksums, c, ws);
                __syncthreads();
            }
        } else if (p == BPH_SCANB) {
            scan_sums_block(I.blocksums, (I.nkeys + 2 + kBatchScanChunk - 1) / kBatchScanChunk, ws);
        } else if (p == BPH_SCANC) {
            // offsets and cursors; the block sort's list emptied
            const int64_t nscan = (I.nkeys + 2 + kBatchScanChunk - 1) / kBatchScanChunk;
            for (int64_t c = c0; c < min(c0 + kBatchChunks, nscan); ++c) {
                scan_apply_block(I.count[st.coff], I.nkeys + 2, I.blocksums, c, ws, I.cursor);
                __syncthreads();
            }
            if (li == 0 && threadIdx.x == 0) I.bigseg[0] = 0;
        } else if (p == BPH_SCATTER) {
            const BatchSort a = sort_of(I, st);
            const int64_t nc = (I.n + kBatchScatterChunk - 1) / kBatchScatterChunk;
            for (int64_t c = c0; c < min(c0 + kBatchChunks, nc); ++c) scatter_pairs_block(a, c);
        } else if (p == BPH_SEG) {
            const BatchSort a = sort_of(I, st);
            const int64_t nc = (I.nkeys + 1 + kBatchSegChunk - 1) / kBatchSegChunk;
            for (int64_t c = c0; c < min(c0 + kBatchChunks, nc); ++c) {
                segments_block(a, c, reinterpret_cast<int32_t(*)[kSegStage]>(smem_raw),
                               reinterpret_cast<int32_t(*)[kSegStage]>(smem_raw + kSegThreads / 32 * kSegStage * 4));
                __syncwarp();
            }
        } else if (p == BPH_ZERO) {
            // the deposit and the next sort's counts zeroed; then (sorted
            // steps) the block sort of long segments
            const int64_t ndep = I.ncell * 4, ncnt = I.nkeys + 2;
            const int64_t nz = (max(ndep, ncnt) + kBatchZeroChunk - 1) / kBatchZeroChunk;
            const int64_t nzi = (nz + kBatchChunks - 1) / kBatchChunks;
            if (li < nzi) {
                const int64_t k1 = min((c0 + kBatchChunks) * kBatchZeroChunk, max(ndep, ncnt));
                for (int64_t k = c0 * kBatchZeroChunk + threadIdx.x; k < k1; k += blockDim.x) {
                    if (k < ndep) I.ta.s.dep[k] = 0ull;
                    if (emit && k < ncnt) I.count[st.coff ^ 1][k] = 0;
                }
            } else {
                const BatchSort a = sort_of(I, st);
                big_segments_block(a, (int32_t)(li - nzi), kBatchBigItems, reinterpret_cast<int32_t *>(smem_raw),
                                   reinterpret_cast<int32_t *>(smem_raw + kBigChunk * 4));
            }
        } else if (p == BPH_TILE) {
            // the step's arguments, with this step's store, permutation and
            // count fields, in shared memory
            {
                const uint64_t *src = reinterpret_cast<const uint64_t *>(&I.ta);
                uint64_t *dst = reinterpret_cast<uint64_t *>(sTA);
                for (int k = threadIdx.x; k < (int)(sizeof(TiledArgs<float>) / 8); k += blockDim.x) dst[k] = src[k];
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                TiledArgs<float> &A = *sTA;
                if (sorted) {
                    A.s.s = I.store[st.cur ^ 1];   // read through the permutation
                    A.dst = I.store[st.cur];
                    A.perm = I.pair_src;
                    A.perm_id = I.pair_id;
                } else {
                    A.s.s = I.store[st.cur];
                    A.dst = I.store[st.cur];
                    A.perm = nullptr;
                    A.perm_id = nullptr;
                }
                A.key_off = I.count[st.coff];
                A.emit_keys = emit ? 1 : 0;
                A.key_out = emit ? I.key : nullptr;
                A.count_out = emit ? I.count[st.coff ^ 1] : nullptr;
            }
            __syncthreads();
            const bool in_time = batch_tile<GEOM, FLAT, MODE, TX, TY, TZ>(*sTA, li, I.ntiles, smem_raw);
            if (!in_time) {
                // the gas box did not arrive in time: stop this block; tasks
                // that wait for this one run out of time too
                ok = false;
                break;
            }
        } else {
            // feedback on the gas, and the time of the next step
            if (I.feedback) {
                const int64_t nc = (I.ncell + kBatchFbChunk - 1) / kBatchFbChunk;
                for (int64_t c = c0; c < min(c0 + kBatchChunks, nc); ++c) {
                    const int64_t z = c * kBatchFbChunk + threadIdx.x;
                    if (z < I.ncell)
                        apply_feedback_zone<float>(I.ta.s.g, I.quantum, const_cast<float *>(I.ta.s.gas), I.ta.s.dep, z);
                }
            }
            if (li == 0 && threadIdx.x == 0) advance_time(I.time, I.dt, I.q_om_lx, I.ly, I.sb);
        }
        signal_done(B.done + t);
    }
    if (!ok && threadIdx.x == 0)
        for (int i = 0; i < B.ninst; ++i) atomicOr(&B.inst[i].ta.s.status[ST_FLAGS], DUST_FLAG_TIMEOUT);
}

template <int GEOM, int FLAT, int MODE, int TX, int TY, int TZ>
int batch_persistent_grid(size_t smem)
{
    auto kern = batch_persistent_kernel<GEOM, FLAT, MODE, TX, TY, TZ>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int per_sm = 0, dev = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSlabThreads, smem) != cudaSuccess)
        return 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return per_sm * sms;
}

template <int GEOM, int FLAT, int MODE, int TX, int TY, int TZ>
cudaError_t launch_batch_persistent(const BatchDev &b, size_t smem, int grid, cudaStream_t s)
{
    auto kern = batch_persistent_kernel<GEOM, FLAT, MODE, TX, TY, TZ>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kSlabThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, b);
}

}  // namespace dust
