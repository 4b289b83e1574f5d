// Batched step of many independent instances as one persistent launch
// (instantiated in dust_slab_batch.cu, beside the step kernels of the same
// geometries).
//
// One cooperative launch (every block resident at once) runs all steps of a
// dust_batch_step call for all instances of a batch.  Each step is a
// sequence of phases; a phase is a list of work items over the instances
// (a chunk of one instance's key counts, grains, keys or zones, or one of its
// tiles) that the blocks take in turn, and a grid barrier separates the
// phases:
//
//   sort (steps s with s % sort_interval == 0):
//     scan A   chunk sums of the key counts the previous step predicted
//     scan B   exclusive scan of the chunk sums, one block per instance
//     scan C   offsets inside each chunk, copied to the scatter's cursors
//     scatter  (id, source) pairs to their key segments
//     segments id sort inside each key (warp-staged)
//   zero       the deposit, the next sort's key counts; block sort of long
//              segments
//   tiles      the slab step kernel's tile function (gather, push, deposit,
//              next keys, and the sort's gather through the permutation)
//   feedback   the deposit applied to the gas; time advanced
//
// Every phase runs the same device functions as the per-context kernels, on
// the same buffers, in the same order per instance, so a batch gives the
// grains, gas and deposit of its instances stepped one at a time, bit for
// bit.  The grid barrier waits a bounded time (wait_ns); when it runs out the
// kernel raises DUST_FLAG_TIMEOUT in every instance's status words and
// returns.
#pragma once

#include <algorithm>

#include "dust_slab.cuh"
#include "dust_sort.cuh"

namespace dust {

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

// Grid barrier over all blocks of the launch, bounded in time.  Thread 0 of
// each block arrives; the last arrival resets the count and bumps the
// generation, the others wait for the generation to change.  Returns false
// (in every thread) when the wait ran out.
__device__ bool grid_barrier(unsigned *bar, unsigned nblocks, unsigned long long limit_ns)
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __syncthreads();
    int ok = 1;
    if (threadIdx.x == 0) {
        volatile unsigned *gen = bar + 1;
        const unsigned g0 = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (*gen == g0) {
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
    // writes of the previous phase (generic proxy) become visible to the
    // next phase's bulk tensor copies (async proxy)
    asm volatile("fence.proxy.async.global;" ::: "memory");
    return ok != 0;
}

// Instance of work item w of phase ph (binary search of the prefix sums).
__device__ __forceinline__ int item_instance(const BatchDev &B, int ph, int w)
{
    const int *pre = B.pre + (size_t)ph * (B.ninst + 1);
    int lo = 0, hi = B.ninst;  // pre[lo] <= w < pre[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] <= w) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int items_of(const BatchDev &B, int ph)
{
    return B.pre[(size_t)ph * (B.ninst + 1) + B.ninst];
}

__device__ __forceinline__ int item_first(const BatchDev &B, int ph, int i)
{
    return B.pre[(size_t)ph * (B.ninst + 1) + i];
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

}  // namespace

template <int GEOM, int FLAT, int MODE>
__global__ void __launch_bounds__(kSlabThreads, 2) batch_persistent_kernel(const BatchDev B)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const unsigned nblk = gridDim.x;
    const unsigned long long lim = B.wait_ns;
    const int K = B.sort_interval;
    unsigned *bar = B.bar;
    bool ok = true;
    auto barrier = [&]() {
        if (ok) ok = grid_barrier(bar, nblk + (unsigned)B.bar_extra, lim);
        return ok;
    };
    int32_t *ws = reinterpret_cast<int32_t *>(smem_raw);  // scan: 32 words
    TiledArgs<float> *sTA = reinterpret_cast<TiledArgs<float> *>(smem_raw + B.ta_offset);
    int *s_item = reinterpret_cast<int *>(smem_raw + B.ta_offset + sizeof(TiledArgs<float>));

    for (int s = 0; s < B.nsteps && ok; ++s) {
        const bool sorted = (s % K) == 0;
        const bool emit = ((s + 1) % K) == 0;
        if (sorted) {
            // ---- scan A: chunk sums of the counts
            for (int w = blockIdx.x; w < items_of(B, BPH_SCAN); w += nblk) {
                const int i = item_instance(B, BPH_SCAN, w);
                const BatchInst &I = B.inst[i];
                const StepState st = state_of(I, s, K);
                scan_reduce_block(I.count[st.coff], I.nkeys + 2, I.blocksums, w - item_first(B, BPH_SCAN, i),
                                  ws);
                __syncthreads();
            }
            if (!barrier()) break;
            // ---- scan B: the chunk sums of each instance
            for (int w = blockIdx.x; w < items_of(B, BPH_INST); w += nblk) {
                const BatchInst &I = B.inst[w];
                scan_sums_block(I.blocksums, (I.nkeys + 2 + kBatchScanChunk - 1) / kBatchScanChunk, ws);
                __syncthreads();
            }
            if (!barrier()) break;
            // ---- scan C: offsets and cursors; the block sort's list emptied
            for (int w = blockIdx.x; w < items_of(B, BPH_SCAN); w += nblk) {
                const int i = item_instance(B, BPH_SCAN, w);
                const BatchInst &I = B.inst[i];
                const StepState st = state_of(I, s, K);
                const int c = w - item_first(B, BPH_SCAN, i);
                scan_apply_block(I.count[st.coff], I.nkeys + 2, I.blocksums, c, ws, I.cursor);
                if (c == 0 && threadIdx.x == 0) I.bigseg[0] = 0;
                __syncthreads();
            }
            if (!barrier()) break;
            // ---- scatter of (id, source) pairs
            for (int w = blockIdx.x; w < items_of(B, BPH_SCATTER); w += nblk) {
                const int i = item_instance(B, BPH_SCATTER, w);
                const BatchInst &I = B.inst[i];
                const BatchSort a = sort_of(I, state_of(I, s, K));
                scatter_pairs_block(a, w - item_first(B, BPH_SCATTER, i));
            }
            if (!barrier()) break;
            // ---- id sort inside each key
            for (int w = blockIdx.x; w < items_of(B, BPH_SEG); w += nblk) {
                const int i = item_instance(B, BPH_SEG, w);
                const BatchInst &I = B.inst[i];
                const BatchSort a = sort_of(I, state_of(I, s, K));
                segments_block(a, w - item_first(B, BPH_SEG, i),
                               reinterpret_cast<int32_t(*)[kSegStage]>(smem_raw),
                               reinterpret_cast<int32_t(*)[kSegStage]>(smem_raw + kSegThreads / 32 * kSegStage * 4));
                __syncwarp();
            }
            if (!barrier()) break;
        }
        // ---- zero the deposit and the next sort's counts; long segments
        for (int w = blockIdx.x; w < items_of(B, BPH_ZERO); w += nblk) {
            const int i = item_instance(B, BPH_ZERO, w);
            const BatchInst &I = B.inst[i];
            const StepState st = state_of(I, s, K);
            const int64_t c = w - item_first(B, BPH_ZERO, i);
            const int64_t ndep = I.ncell * 4, ncnt = I.nkeys + 2;
            for (int64_t k = c * kBatchZeroChunk + threadIdx.x; k < (c + 1) * kBatchZeroChunk; k += blockDim.x) {
                if (k < ndep) I.ta.s.dep[k] = 0ull;
                if (emit && k < ncnt) I.count[st.coff ^ 1][k] = 0;
            }
        }
        if (sorted) {
            for (int w = blockIdx.x; w < B.ninst * kBatchBigItems; w += nblk) {
                const int i = w / kBatchBigItems;
                const BatchInst &I = B.inst[i];
                const BatchSort a = sort_of(I, state_of(I, s, K));
                big_segments_block(a, w % kBatchBigItems, kBatchBigItems, reinterpret_cast<int32_t *>(smem_raw),
                                   reinterpret_cast<int32_t *>(smem_raw + kBigChunk * 4));
                __syncthreads();
            }
        }
        if (!barrier()) break;
        // ---- step: the tiles of every instance, the heaviest instances'
        // tiles first, each block taking the next tile from a counter
        const int ntile_items = items_of(B, BPH_TILE);
        for (;;) {
            __syncthreads();
            if (threadIdx.x == 0) *s_item = atomicAdd(&B.ctr[s], 1);
            __syncthreads();
            const int w = *s_item;
            if (w >= ntile_items) break;
            const int j = item_instance(B, BPH_TILE, w);
            const int i = B.tile_order[j];
            const BatchInst &I = B.inst[i];
            const StepState st = state_of(I, s, K);
            // the step's arguments, with this step's store, permutation and
            // count fields, in shared memory
            {
                const uint64_t *src = reinterpret_cast<const uint64_t *>(&I.ta);
                uint64_t *dst = reinterpret_cast<uint64_t *>(sTA);
                for (int k = threadIdx.x; k < (int)(sizeof(TiledArgs<float>) / 8); k += blockDim.x) dst[k] = src[k];
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                TiledArgs<float> &T = *sTA;
                if (sorted) {
                    T.s.s = I.store[st.cur ^ 1];   // read through the permutation
                    T.dst = I.store[st.cur];
                    T.perm = I.pair_src;
                    T.perm_id = I.pair_id;
                } else {
                    T.s.s = I.store[st.cur];
                    T.dst = I.store[st.cur];
                    T.perm = nullptr;
                    T.perm_id = nullptr;
                }
                T.key_off = I.count[st.coff];
                T.emit_keys = emit ? 1 : 0;
                T.key_out = emit ? I.key : nullptr;
                T.count_out = emit ? I.count[st.coff ^ 1] : nullptr;
            }
            __syncthreads();
            const bool in_time = slab_tile<GEOM, FLAT, MODE>(*sTA, w - item_first(B, BPH_TILE, j), I.ntiles,
                                                             smem_raw, true);
            // every thread is done with the arguments before the next copy
            __syncthreads();
            if (!in_time) {
                // the gas box did not arrive in time: stop this block (the
                // others run out at the next barrier)
                ok = false;
                break;
            }
        }
        if (!barrier()) break;
        // ---- feedback on the gas, and the time of the next step
        for (int w = blockIdx.x; w < items_of(B, BPH_FB); w += nblk) {
            const int i = item_instance(B, BPH_FB, w);
            const BatchInst &I = B.inst[i];
            const int c0 = w - item_first(B, BPH_FB, i);
            if (I.feedback) {
                const int64_t c = (int64_t)c0 * blockDim.x + threadIdx.x;
                if (c < I.ncell) apply_feedback_zone<float>(I.ta.s.g, I.quantum, const_cast<float *>(I.ta.s.gas),
                                                            I.ta.s.dep, c);
            }
            if (c0 == 0 && threadIdx.x == 0) advance_time(I.time, I.dt, I.q_om_lx, I.ly, I.sb);
        }
        if (!barrier()) break;
    }
    if (!ok && threadIdx.x == 0)
        for (int i = 0; i < B.ninst; ++i) atomicOr(&B.inst[i].ta.s.status[ST_FLAGS], DUST_FLAG_TIMEOUT);
}

template <int GEOM, int FLAT, int MODE>
int batch_persistent_grid(size_t smem)
{
    auto kern = batch_persistent_kernel<GEOM, FLAT, MODE>;
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

template <int GEOM, int FLAT, int MODE>
cudaError_t launch_batch_persistent(const BatchDev &b, size_t smem, int grid, cudaStream_t s)
{
    auto kern = batch_persistent_kernel<GEOM, FLAT, MODE>;
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
