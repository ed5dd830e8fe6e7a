// persist.cuh -- the persistent fused-update iteration: many 3MG iterations of
// every plain volume of a context in one cooperative launch.
//
// The fused-update iteration of plain volumes (no slabs) is two passes per
// iteration (lazy.cuh): the gradient pass (Master step (2) applied lazily, the
// Worker's gradient step (3) and the objective, Section 3.1 Eq. "crit") and the
// curvature pass (the sums of D^T A D and D^T grad f, Eq. "maj", and in its
// last CTA the 2x2 solve of Eq. "minimizer").  k_persist runs `iters` such
// iterations in one launch: a grid of CTAs that are all resident at once (a
// cooperative launch sized from the occupancy) takes the work items of a pass
// from a queue (one atomic counter per pass), then waits at a grid-wide
// barrier before the next pass.  The per-item code is the one of the separate
// launches (gradlazy_item, curvature_item), every partial sum lands in the row
// of its item and the last CTA of a pass sums the rows in item order, so the
// iterates are the bits the two-launch iteration produces.
//
// Volumes stop inside the launch: the gradient pass's finish sets a volume's
// stop flag, and every later item of that volume only takes its ticket.  No
// host round trip re-plans the work lists between iterations.
//
// Every wait is bounded: the grid barrier gives up after the context's wait
// limit, sets ST_TIMEOUT in the status word and every CTA leaves at the next
// barrier; a CTA whose item ran out of time takes no further item.
#pragma once
#include "lazy.cuh"

namespace bd3mg {

// Device words of one persistent launch, zeroed before it: [0] arrivals at the
// grid barrier, [1] barrier generation, [2] item queue of the gradient pass,
// [3] item queue of the curvature pass.
constexpr int PERSIST_WORDS = 4;

struct PersistArgs {
    KArgs g;                  // fused-update gradient pass over every volume's items
    KArgs c;                  // curvature pass
    unsigned int *words;      // PERSIST_WORDS
    int iters;
};

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier of the nblocks CTAs of a cooperative launch.  The pass's
// global writes (generic proxy) are made visible to the next pass's TMA reads
// (async proxy) on both sides of the release/acquire pair.  True (all threads
// of the CTA) when the next pass may start: the barrier completed within
// limit_ns and no CTA has reported ST_TIMEOUT.
__device__ __forceinline__ bool grid_barrier(unsigned int *words, unsigned int nblocks, unsigned long long limit_ns,
                                             int *status) {
    __shared__ int go;
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned int gen = ld_acquire_u32(words + 1);
        __threadfence();
        bool ok = true;
        if (atomicAdd(words, 1u) == nblocks - 1) {
            words[0] = 0u;                       // ordered before the release below
            __threadfence();
            atomicAdd(words + 1, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (ld_acquire_u32(words + 1) == gen) {
                if (global_ns() - t0 > limit_ns) {
                    ok = false;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        asm volatile("fence.proxy.async.global;" ::: "memory");
        if (!ok) atomicOr(status, ST_TIMEOUT);
        go = ok && (*reinterpret_cast<volatile int *>(status) & ST_TIMEOUT) == 0;
    }
    __syncthreads();
    return go != 0;
}

// Next work item of a pass for this CTA, or -1 when the pass's queue is empty.
// The queue counter only grows: in iteration k the pass hands out the values
// base .. base + nitems - 1 as items and one more value per CTA (each CTA's
// last take), so base = k (nitems + gridDim.x).
__device__ __forceinline__ int take_item(unsigned int *queue, unsigned int base, int nitems) {
    __shared__ int got;
    __syncthreads();                             // every thread has read the previous take
    if (threadIdx.x == 0) got = (int)(atomicAdd(queue, 1u) - base);
    __syncthreads();
    return got < nitems ? got : -1;
}

// Host-set fault injection (Shared::fault): CTA 0 of a persistent launch leaves
// without arriving at its first grid barrier, so every other CTA's barrier wait
// runs out and the host reads ST_TIMEOUT.
constexpr int FAULT_SKIP_ARRIVE = 2;

template <int R, int RZ, bool BF, int PM>
__global__ void __launch_bounds__(NT, 2) k_persist(const __grid_constant__ PersistArgs p) {
    constexpr int RPT = BF ? 2 : 1;              // curvature rows per thread: the 16-row FP32 / 32-row BF16 tiles
    unsigned int *w = p.words;
    const unsigned int nb = gridDim.x;
    const unsigned long long limit = p.g.sh->wait_ns;
    int *status = p.g.sh->status;
    for (int k = 0; k < p.iters; ++k) {
        bool ok = true;
        const unsigned int bg = (unsigned int)k * (unsigned int)(p.g.nitems + (int)nb);
        for (int it; ok && (it = take_item(w + 2, bg, p.g.nitems)) >= 0;)
            ok = gradlazy_item<R, RZ, BF, PM, true>(p.g, it);
        if (p.g.sh->fault == FAULT_SKIP_ARRIVE && blockIdx.x == 0) return;
        if (!grid_barrier(w, nb, limit, status)) return;
        const unsigned int bc = (unsigned int)k * (unsigned int)(p.c.nitems + (int)nb);
        for (int it; ok && (it = take_item(w + 3, bc, p.c.nitems)) >= 0;)
            ok = curvature_item<R, RZ, BF, PM, RPT, true>(p.c, it);
        if (!grid_barrier(w, nb, limit, status)) return;
    }
}

}  // namespace bd3mg
