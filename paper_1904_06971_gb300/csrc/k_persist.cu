// Persistent quadrature over the patches of a batch: the stage bodies of
// quad_bodies.cuh run from one launch per (dimension, degree, arithmetic).
#include "quad_bodies.cuh"

namespace iga {

// ---------------------------------------------------------------------------
// Persistent quadrature over the patches of a batch (one launch per degree,
// dimension and arithmetic).  The work items are the blocks of the stage
// launches of every patch, in stage-major order (all Z-half-0 blocks, all
// Z-half-1 blocks, all Y, all X).  A block claims `chunk` consecutive items
// from a device counter, waits until the previous stage of the item's patch is
// complete (completion counters, bounded wait), runs the stage body with the
// item's block index and counts the item done.  Items are claimed in order and
// depend only on items with smaller indices, so the smallest unfinished item
// can always run: the launch needs no co-residency of its blocks.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait (one thread) until c0 >= n0 and c1 >= n1 (c1 may be null).  Gives up when
// another block raised ctl->abort, or after limit_ns of the global timer or
// 2^24 polls: then sets ctl->status and ctl->abort and returns false.
__device__ bool persist_wait(const unsigned* c0, unsigned n0, const unsigned* c1, unsigned n1, PersistCtl* ctl,
                             long long limit_ns)
{
    const unsigned long long t0 = global_ns();
    unsigned sleep_ns = 32;
    for (int it = 0; it < (1 << 24); ++it) {
        if (ld_acquire_u32(c0) >= n0 && (!c1 || ld_acquire_u32(c1) >= n1)) return true;
        if (*reinterpret_cast<volatile int*>(&ctl->abort)) return false;
        if ((long long)(global_ns() - t0) > limit_ns) break;
        __nanosleep(sleep_ns);
        if (sleep_ns < 1024) sleep_ns *= 2;
    }
    atomicExch(&ctl->status, 1);
    atomicExch(&ctl->abort, 1);
    return false;
}

template <class Pol, int P, int DIM>
__global__ void __launch_bounds__(kBlock) k_persist(const PersistWork* __restrict__ works,
                                                    const PersistSeg* __restrict__ segs, int nseg, int64_t total,
                                                    int chunk, PersistCtl* ctl, unsigned* done, long long limit_ns)
{
    __shared__ int64_t s_first;
    __shared__ int s_go;
    for (;;) {
        __syncthreads();                 // s_first / s_go of the previous round are no longer read
        if (threadIdx.x == 0) {
            const bool stop = *reinterpret_cast<volatile int*>(&ctl->abort) != 0;
            s_first = stop ? total : (int64_t)atomicAdd(&ctl->next, (unsigned long long)chunk);
        }
        __syncthreads();
        const int64_t first = s_first;
        if (first >= total) return;
        const int64_t last = (first + chunk < total) ? first + chunk : total;
        for (int64_t it = first; it < last; ++it) {
            int lo = 0, hi = nseg - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (segs[mid].first <= it) lo = mid;
                else hi = mid - 1;
            }
            const int stage = segs[lo].stage;
            const PersistWork& w = works[segs[lo].work];
            const int64_t blk = it - segs[lo].first;
            if (threadIdx.x == 0) {
                bool go = true;
                if (stage == 3 && DIM == 3)
                    go = persist_wait(done + w.done0, (unsigned)w.nb[1], done + w.done0 + 1, (unsigned)w.nb[1], ctl,
                                      limit_ns);
                else if (stage == 4)
                    go = persist_wait(done + w.done0 + 2, (unsigned)w.nb[2], nullptr, 0u, ctl, limit_ns);
                s_go = go ? 1 : 0;
            }
            __syncthreads();
            if (!s_go) return;
            if constexpr (DIM == 3) {
                if (stage == 1) stage_z_body<Pol, P, 0>(w.g, w.T, w.bs, w.scratch, blk);
                else if (stage == 2) stage_z_body<Pol, P, 1>(w.g, w.T, w.bs, w.scratch, blk);
            }
            if (stage == 3) stage_y_body<Pol, P, DIM>(w.g, w.T, w.bs, w.scratch, blk);
            else if (stage == 4)
                stage_x_body<Pol, P, DIM, kLinesX>(w.g, w.T, w.bs, w.scratch, w.ell, w.ell_f32, w.N, w.samples, 0, blk);
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(done + w.done0 + (stage - 1), 1u);
            }
        }
    }
}

template <class Pol, int P>
static const void* persist_fn(int dim)
{
    return dim == 3 ? (const void*)k_persist<Pol, P, 3> : (const void*)k_persist<Pol, P, 2>;
}

static const void* persist_kernel(int dim, int p, int arith)
{
#define IGA_PERSIST_P(POL)                                   \
    switch (p) {                                             \
    case 1: return persist_fn<POL, 1>(dim);                  \
    case 2: return persist_fn<POL, 2>(dim);                  \
    case 3: return persist_fn<POL, 3>(dim);                  \
    case 4: return persist_fn<POL, 4>(dim);                  \
    case 5: return persist_fn<POL, 5>(dim);                  \
    default: return nullptr;                                 \
    }
    if (dim != 2 && dim != 3) return nullptr;
    switch (arith) {
    case kArithF32: IGA_PERSIST_P(PolF32)
    case kArithDF: IGA_PERSIST_P(PolDF)
    case kArithF64: IGA_PERSIST_P(PolF64)
    default: return nullptr;
    }
#undef IGA_PERSIST_P
}

int persist_blocks_per_sm(int dim, int p, int arith)
{
    const void* fn = persist_kernel(dim, p, arith);
    if (!fn) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, kBlock, 0) != cudaSuccess) return 0;
    return n;
}

cudaError_t launch_persist(int dim, int p, int arith, const PersistWork* works, const PersistSeg* segs, int nseg,
                           int64_t total, int chunk, int grid, PersistCtl* ctl, unsigned* done, long long limit_ns,
                           cudaStream_t s)
{
    const void* fn = persist_kernel(dim, p, arith);
    if (!fn || grid < 1 || chunk < 1 || nseg < 1) return cudaErrorInvalidValue;
    void* args[] = {(void*)&works, (void*)&segs, (void*)&nseg, (void*)&total, (void*)&chunk, (void*)&ctl, (void*)&done,
                    (void*)&limit_ns};
    launch_begin(K_PERSIST, s);
    cudaError_t e = cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(kBlock), args, 0, s);
    launch_end(K_PERSIST, s);
    return e;
}

}  // namespace iga
