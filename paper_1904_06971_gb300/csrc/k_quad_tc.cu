// K3 stage X on the tensor cores (tcgen05, sm_103a), for FP32 values.
//
// Stage X contracts direction 0 (k_quad.cu): for a line (pair3, pair2) of the
// stage-Y output T2 and a row i0 whose stencil stays among cardinal B-splines,
//     A_row[delta0] = sum_g sum_t T2[g][line][(i0 - p - elo) Q + t] X_card[delta0][t][pat(g)],
// t = a Q + r over the (p+1)^2 Gauss points of supp(B_i0); the pair weights
// X_card are the same for every cardinal row (translation invariance, Sec. 2.2).
// For 128 lines at a time this is a product of an MN-major A (lines x Gauss
// points, a sliding window per row i0) and a K-major B (Gauss points x offsets,
// 2p+1 <= 16 columns): one tcgen05 MMA chain per row into its own 16 columns of
// tensor memory.  The window of row i0 starts Q rows after that of row i0 - 1,
// so one shared-memory tile of the Gauss points of a chunk of rows serves all
// of them without copies (the descriptor start moves by whole 16-byte K rows).
//
// FP32 accuracy from BF16 operands: every FP32 value x is split into three
// BF16 parts x0 + x1 + x2 (each the rounded remainder of the previous ones, 24
// significand bits in all); the six partial products of total order <= 2
// (a0 b0, a0 b1, a1 b0, a0 b2, a1 b1, a2 b0) accumulate in FP32 in tensor
// memory.  The dropped products are below 2^-24 of the terms, the size of the
// FP32 rounding of the CUDA-core kernel they replace.
//
// Rows outside the cardinal range, one-row sample boxes and every other
// arithmetic stay on the CUDA-core kernel of k_quad.cu.
#include <cuda_bf16.h>

#include "arith.cuh"
#include "iga_internal.cuh"
#include "tc_ptx.cuh"

namespace iga {

namespace {

constexpr int kTcThreads = 512;         // 16 warps: all copy and split, the lanes 0 of the first ones issue MMAs
constexpr int kTcLines = 128;           // MMA M: lines per block
constexpr int kTcN = 16;                // MMA N: offsets delta0 (2p + 1 <= 11 used)
constexpr int kTcSlices = 3;            // BF16 parts per FP32 value
constexpr int kTcWaitIter = 1 << 22;    // polls of an mbarrier before the kernel gives up

// Tile shapes per degree.  A "job" is one (chunk of C rows i0, T2 group) pair:
// its Gauss points (ROWS per line) are copied asynchronously into a raw FP32
// tile, split into the BF16 tile, and consumed by the MMAs of the chunk's rows.
// Raw tiles, BF16 tiles and tensor-memory blocks are all double-buffered.
template <int P>
struct TcShape {
    static constexpr int Q = P + 1, W = 2 * P + 1, TT = Q * Q;
    static constexpr int KW = (TT + 15) / 16 * 16;           // K rows of one window (zero weights beyond TT)
    static constexpr int KSTEPS = KW / 16;
    static constexpr int C = (P >= 5) ? 4 : 5;               // rows i0 per chunk
    static constexpr int ROWS = (C - 1) * Q + KW;            // Gauss points of a chunk's tile
    static constexpr int A_SLICE = 16 * ROWS * 16;           // bytes of one BF16 part of the A tile (16 line groups)
    static constexpr int A_BUF = kTcSlices * A_SLICE;        // bytes of one BF16 tile
    static constexpr int RAW = kTcLines * ROWS * 4;          // bytes of one raw FP32 tile
    static constexpr int NB = kTcSlices * kTcN;              // B rows of one pattern: its three parts side by side
    static constexpr int B_GROUP = NB * KW * 2;              // bytes of one pattern's B
    static constexpr int B_BYTES = 4 * B_GROUP;
    static constexpr int SMEM = 2 * A_BUF + 2 * RAW + B_BYTES + 128;
    static constexpr int TBLOCK = C * NB;                    // tensor-memory columns of one chunk (three level blocks a row)
    static constexpr int TMEM_COLS = (2 * TBLOCK <= 128) ? 128 : (2 * TBLOCK <= 256 ? 256 : 512);
    static_assert(SMEM <= 227 * 1024, "tile does not fit in shared memory");
    static_assert(2 * TBLOCK <= 512, "chunk does not fit in tensor memory");
};

// The three BF16 parts of x (round to nearest at each step; the remainders are exact in FP32).
__device__ __forceinline__ void split3(float x, __nv_bfloat16& a0, __nv_bfloat16& a1, __nv_bfloat16& a2)
{
    a0 = __float2bfloat16_rn(x);
    const float r1 = __fsub_rn(x, __bfloat162float(a0));
    a1 = __float2bfloat16_rn(r1);
    const float r2 = __fsub_rn(r1, __bfloat162float(a1));
    a2 = __float2bfloat16_rn(r2);
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

}  // namespace

// Set when a tensor-core stage gave up waiting for its MMAs (never expected);
// the rows it did not finish are written as NaN.
__device__ int g_tc_status = 0;

// One block per 128 consecutive lines (pair3, pair2) of box b; the rows i0 in
// [i0_lo, i0_hi] (all cardinal) in chunks of C rows, four jobs (T2 groups =
// direction-0 patterns) per chunk.  Per job: the block's threads copy the
// job's Gauss points of their lines asynchronously into a raw FP32 tile (the
// copy of the next job is in flight while this one is processed), split them
// into three BF16 parts in an MN-major tile (16 groups of 8 lines, one 16-byte
// row per Gauss point), and lane 0 of warp w issues the MMAs of chunk row w:
// per K step and A part i one MMA against the B parts 0 .. 2 - i of the
// pattern side by side (K-major, 16 offset columns each, N = 16 (3 - i)), its
// D starting at the row's level block i, so part j lands in block i + j (the
// three blocks of a row are added in the epilogue).  One MMA thus reads its A
// part from shared memory once for all its B parts.  mbarriers tell
// when a BF16 tile's MMAs are done; after the first job of chunk k has been
// issued, the rows of chunk k - 1 are read out of the other tensor-memory
// block and written to the stencil-ELL values.
template <int P, int DIM>
__global__ void __launch_bounds__(kTcThreads, 1)
k_stage_x_tc(Geo g, Tables T, Box b, int i0_lo, int i0_hi, const double* scratch, float* ell, int64_t N)
{
    using Sh = TcShape<P>;
    constexpr int Q = Sh::Q, W = Sh::W, TT = Sh::TT, KW = Sh::KW, C = Sh::C, ROWS = Sh::ROWS;
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    unsigned char* sA = tc_smem;                                         // [2][part 3][line group 16][ROWS][16 B]
    float* sR = reinterpret_cast<float*>(tc_smem + 2 * Sh::A_BUF);       // [2][line 128][ROWS]
    unsigned char* sB = tc_smem + 2 * Sh::A_BUF + 2 * Sh::RAW;           // [group 4][part x 16 + n: 6 groups of 8][K block][128 B]
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + Sh::B_BYTES);      // [0..1] BF16 tile consumed, [2] drain
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    const int64_t G0 = (int64_t)b.E[0] * Q;
    const int64_t P3 = (DIM == 3) ? (int64_t)b.R[2] * W : 1;
    const int64_t P2 = (int64_t)b.R[1] * W;
    const int64_t total = P3 * P2;                    // lines of the box
    const int64_t line0 = (int64_t)blockIdx.x * kTcLines;
    const float* T2 = reinterpret_cast<const float*>(scratch + b.t2_off);
    const int64_t gs = total * G0;                    // group stride of T2
    const int nchunks = (i0_hi - i0_lo) / C + 1;
    const int jobs = 4 * nchunks;

    // asynchronous copy of job j's Gauss points into raw tile j & 1 (zeros beyond the box)
    auto issue_copy = [&](int j) {
        const int c0 = i0_lo + (j >> 2) * C, gq = j & 3;
        const int64_t row0 = (int64_t)(c0 - P - b.elo[0]) * Q;
        const float* src = T2 + (int64_t)gq * gs;
        float* dst = sR + (size_t)(j & 1) * (kTcLines * ROWS);
        for (int idx = tid; idx < kTcLines * ROWS; idx += kTcThreads) {
            const int l = idx / ROWS, r = idx - l * ROWS;
            const int64_t line = line0 + l, gp = row0 + r;
            const bool valid = line < total && gp < G0;
            tc::cp_async4(dst + idx, valid ? src + line * G0 + gp : T2, valid);
        }
        tc::cp_async_commit();
    };
    issue_copy(0);

    // B: cardinal pair weights of direction 0 in three BF16 parts, one K-major
    // [3 x 16 offsets x KW Gauss points] matrix per pattern, part j in rows 16 j .. 16 j + 15
    // (zero beyond 2p+1 and TT)
    const float* Xc = reinterpret_cast<const float*>(T.Xs[0]) + (int64_t)(2 * P) * W * TT * 4;
    for (int idx = tid; idx < 4 * kTcN * KW; idx += kTcThreads) {
        const int gq = idx / (kTcN * KW), n = (idx / KW) % kTcN, k = idx % KW;
        const int pat = 3 - gq;                       // T2 group 0: pattern 11, 1: 10, 2: 01, 3: 00
        const float x = (n < W && k < TT) ? Xc[((int64_t)n * TT + k) * 4 + pat] : 0.f;
        __nv_bfloat16 xp[3];
        split3(x, xp[0], xp[1], xp[2]);
        __nv_bfloat16* base = reinterpret_cast<__nv_bfloat16*>(sB + (size_t)gq * Sh::B_GROUP);
#pragma unroll
        for (int jd = 0; jd < 3; ++jd) {
            const int r = jd * kTcN + n;
            base[((r >> 3) * (KW / 8) + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7)] = xp[jd];
        }
    }
    if (tid == 0) {
        // every warp's lane 0 issues MMAs and commits to these barriers
        tc::bar_init(&bars[0], kTcThreads / 32);
        tc::bar_init(&bars[1], kTcThreads / 32);
        tc::bar_init(&bars[2], kTcThreads / 32);
        tc::fence_bar_init();
    }
    if (warp == 0) tc::tmem_alloc(tmem_slot, Sh::TMEM_COLS);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    // this thread's output line (epilogue): warp w reads tensor-memory lanes 32 (w % 4) ..
    const int q4 = warp & 3, quarter = warp >> 2;
    const int64_t my_line = line0 + q4 * 32 + lane;
    int64_t rowbase = 0;
    int slot0 = 0;
    if (my_line < total) {
        const int64_t pair3 = my_line / P2, pair2 = my_line - pair3 * P2;
        const int i1 = b.rlo[1] + (int)(pair2 / W), d1 = (int)(pair2 % W);
        const int i2 = (DIM == 3) ? b.rlo[2] + (int)(pair3 / W) : 0;
        const int d2 = (DIM == 3) ? (int)(pair3 % W) : 0;
        rowbase = (int64_t)g.m[0] * (i1 + (int64_t)g.m[1] * i2);
        slot0 = W * (d1 + W * d2);
    }
    // rows of chunk k out of tensor-memory block k & 1, once its last job's MMAs are done
    auto epilogue = [&](int k) -> bool {
        const int last = 4 * k + 3;
        const bool ok = __syncthreads_and(warp == 0 ? tc::bar_wait(&bars[last & 1], (uint32_t)((last >> 1) & 1), kTcWaitIter)
                                                    : true) != 0;
        if (!ok) return false;
        tc::fence_after_sync();
        const int c0 = i0_lo + k * C, nc = min(C, i0_hi - c0 + 1);
        const uint32_t tb = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)((k & 1) * Sh::TBLOCK);
        for (int c = quarter; c < nc; c += kTcThreads / 128) {
            float v0[16], v1[16], v2[16];
            tc::tmem_ld16(tb + (uint32_t)(c * Sh::NB), v0);
            tc::tmem_ld16(tb + (uint32_t)(c * Sh::NB + kTcN), v1);
            tc::tmem_ld16(tb + (uint32_t)(c * Sh::NB + 2 * kTcN), v2);
            if (my_line < total) {
                const int64_t row = c0 + c + rowbase;
#pragma unroll
                for (int dd = 0; dd < W; ++dd) ell[(int64_t)(slot0 + dd) * N + row] = v0[dd] + (v1[dd] + v2[dd]);
            }
        }
        tc::fence_before_sync();
        return true;
    };

    const uint32_t sA_addr = tc::smem_addr(sA), sB_addr = tc::smem_addr(sB);
    bool ok = true;
    int done_chunks = 0;              // chunks whose rows are written
    for (int j = 0; j < jobs; ++j) {
        const int k = j >> 2, gq = j & 3, buf = j & 1;
        const int c0 = i0_lo + k * C, nc = min(C, i0_hi - c0 + 1);
        // raw tile (j + 1) & 1 was last read by job j - 1, whose split ended in a barrier
        if (j + 1 < jobs) {
            issue_copy(j + 1);
            tc::cp_async_wait<1>();
        } else {
            tc::cp_async_wait<0>();
        }
        // BF16 tile buf was last read by the MMAs of job j - 2
        // (one warp polls the mbarrier; the others wait at the block barrier without taking issue slots)
        const bool wok = (j >= 2 && warp == 0) ? tc::bar_wait(&bars[buf], (uint32_t)(((j >> 1) - 1) & 1), kTcWaitIter) : true;
        ok = __syncthreads_and(wok) != 0;            // also makes every thread's copies of job j visible
        if (!ok) break;
        const float* raw = sR + (size_t)buf * (kTcLines * ROWS);
        unsigned char* tile = sA + (size_t)buf * Sh::A_BUF;
        for (int item = tid; item < 16 * ROWS; item += kTcThreads) {
            const int lg = item / ROWS, r = item - lg * ROWS;
            const float* rp = raw + (size_t)lg * 8 * ROWS + r;
            uint32_t w0[4], w1[4], w2[4];
#pragma unroll
            for (int l = 0; l < 8; l += 2) {
                __nv_bfloat16 a0, a1, a2, b0, b1, b2;
                split3(rp[l * ROWS], a0, a1, a2);
                split3(rp[(l + 1) * ROWS], b0, b1, b2);
                w0[l / 2] = pack2(a0, b0);
                w1[l / 2] = pack2(a1, b1);
                w2[l / 2] = pack2(a2, b2);
            }
            const size_t off = ((size_t)lg * ROWS + r) * 16;
            *reinterpret_cast<uint4*>(tile + off) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
            *reinterpret_cast<uint4*>(tile + Sh::A_SLICE + off) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
            *reinterpret_cast<uint4*>(tile + 2 * Sh::A_SLICE + off) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
        }
        tc::fence_async_smem();
        __syncthreads();
        // MMAs: lane 0 of warp c issues those of chunk row c (a row's chain stays in one thread, so its
        // accumulation order is fixed); descriptors advance by whole 16-byte rows
        if (lane == 0) {
            tc::fence_after_sync();
            const uint64_t a0 = tc::sdesc(sA_addr + (uint32_t)(buf * Sh::A_BUF), 128, ROWS * 16);
            const uint64_t b0 = tc::sdesc(sB_addr + (uint32_t)(gq * Sh::B_GROUP), 128, (KW / 8) * 128);
            const uint32_t d_base = tmem + (uint32_t)((k & 1) * Sh::TBLOCK);
            for (int c = warp; c < nc; c += kTcThreads / 32) {
#pragma unroll
                for (int ks = 0; ks < Sh::KSTEPS; ++ks) {
                    const uint64_t arow = (uint64_t)(c * Q + ks * 16);
#pragma unroll
                    for (int i = 0; i < kTcSlices; ++i) {
                        // A part i times B parts 0 .. 2 - i: products of order i + j <= 2, part j into level block i + j
                        const uint32_t idesc = tc::idesc_bf16_f32(kTcLines, kTcN * (kTcSlices - i), 1, 0);
                        const uint64_t ad = a0 + (uint64_t)(i * Sh::A_SLICE / 16) + arow;
                        const uint64_t bd = b0 + (uint64_t)(ks * 256 / 16);
                        tc::mma_bf16(d_base + (uint32_t)(c * Sh::NB + i * kTcN), ad, bd, idesc, (gq | ks | i) ? 1u : 0u);
                    }
                }
            }
            tc::commit(&bars[buf]);
        }
        if (gq == 0 && k >= 1) {
            if (!epilogue(k - 1)) { ok = false; break; }
            done_chunks = k;
        }
    }
    if (ok) {
        ok = epilogue(nchunks - 1);
        if (ok) done_chunks = nchunks;
    }
    if (!ok) {
        // give up: mark the status, let the copies and every issued MMA drain, NaN the rows not written
        tc::cp_async_wait<0>();
        if (tid == 0) atomicOr(&g_tc_status, 1);
        if (lane == 0) tc::commit(&bars[2]);
        tc::bar_wait(&bars[2], 0u, kTcWaitIter);
        if (quarter == 0 && my_line < total)
            for (int i0 = i0_lo + done_chunks * C; i0 <= i0_hi; ++i0)
                for (int dd = 0; dd < W; ++dd)
                    ell[(int64_t)(slot0 + dd) * N + rowbase + i0] = __int_as_float(0x7fc00000);
    }
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, Sh::TMEM_COLS);
}

// ---------------------------------------------------------------------------
// FP64 values: exact BF16 digit products (the FP64 accuracy of double-float
// stage X, on the tensor cores).
//
// Every T2 value of a line (double-float) is scaled by a power of two to
// |alpha| < 1 -- per line, from the largest exponent stage Y recorded, with the
// four T2 groups balanced by powers of two sigma_g against the pair weights
// they meet -- and written as seven signed base-256 digits alpha = sum_i a_i,
// a_i = (integer of magnitude <= 129) 2^-(7+8i), each exact in BF16.  The pair
// weights (FP64) get the same seven digits per offset column.  A product
// a_i b_j is an integer times 2^-(14+8(i+j)), so the products of one level
// L = i + j <= 3 summed over the K = 4 (p+1)^2 Gauss points of a row stay below
// 2^24 quanta: their FP32 accumulation is exact; every level has its own block
// of tensor memory (the FP32 rounding of levels 4..6 is below 2^-50 of the
// row's terms).  Levels >= 7 and the digits beyond the seventh are dropped
// (below 2^-55).  One MMA takes A digit i against B digits 0 .. 6 - i side by
// side (N = 16 (7 - i)), its D starting at the row's level block i, so digit j
// lands in block i + j: the A digit is read from shared memory once for all of
// them.  The seven blocks are added in double-float, scaled back and rounded
// once to double.
// ---------------------------------------------------------------------------
namespace {

constexpr int kDigits = 7;              // BF16 digits per value (and level blocks of tensor memory per row)

template <int P>
struct Tc64Shape {
    static constexpr int Q = P + 1, W = 2 * P + 1, TT = Q * Q;
    static constexpr int KW = (TT + 15) / 16 * 16;
    static constexpr int KSTEPS = KW / 16;
    static constexpr int C = (P >= 5) ? 1 : 4;               // rows i0 per chunk (NB columns of tensor memory each)
    static constexpr int ROWS = (C - 1) * Q + KW;
    static constexpr int A_SLICE = 16 * ROWS * 16;
    static constexpr int A_BUF = kDigits * A_SLICE;          // one digit tile (two alternate)
    static constexpr int NB = kDigits * kTcN;                // B rows of one pattern: its seven digits side by side
    static constexpr int B_GROUP = NB * KW * 2;
    static constexpr int B_BYTES = 4 * B_GROUP;
    static constexpr int SMALL = kTcLines * 4 * 4 + kTcLines * 4 + kTcN * 4 + 64;   // scales, exponents, barriers
    static constexpr int SMEM = 2 * A_BUF + B_BYTES + SMALL;
    static constexpr int TMEM_COLS = 512;
    static_assert(C * NB <= TMEM_COLS, "chunk does not fit in tensor memory");
    static_assert(SMEM <= 227 * 1024, "tile does not fit in shared memory");
};

__device__ __forceinline__ float pow2f(int k)
{
    k = max(-126, min(127, k));
    return __int_as_float((127 + k) << 23);
}

}  // namespace

// Group shifts sigma_g = E(max |X_g|) - E(max |X_0|) of the cardinal pair
// weights of direction 0 (pattern of T2 group g: 11, 10, 01, 00), E = binary
// exponent; one block.
__global__ void k_tc_group_shift(const double* Xcard, int W, int TT, int* gshift)
{
    __shared__ int mx[4];
    if (threadIdx.x < 4) mx[threadIdx.x] = -100000;
    __syncthreads();
    for (int idx = threadIdx.x; idx < 4 * W * TT; idx += blockDim.x) {
        const int gq = idx / (W * TT), r = idx % (W * TT);
        const double x = Xcard[(int64_t)r * 4 + (3 - gq)];
        if (x != 0.0) atomicMax(&mx[gq], ilogb(x));
    }
    __syncthreads();
    if (threadIdx.x < 4) gshift[threadIdx.x] = (mx[threadIdx.x] > -100000 && mx[0] > -100000) ? mx[threadIdx.x] - mx[0] : 0;
}

cudaError_t launch_tc_group_shift(const Geo& g, const Tables& T, int* gshift, cudaStream_t s)
{
    const int W = 2 * g.p + 1, TT = (g.p + 1) * (g.p + 1);
    if (g.m[0] < 4 * g.p + 1) return cudaMemsetAsync(gshift, 0, 4 * sizeof(int), s);
    launch_begin(K_STAGE_X_TC, s);
    k_tc_group_shift<<<1, 256, 0, s>>>(T.X[0] + (int64_t)(2 * g.p) * W * TT * 4, W, TT, gshift);
    launch_end(K_STAGE_X_TC, s);
    return cudaGetLastError();
}

// One block per 128 lines of box b, rows i0 in [i0_lo, i0_hi] (cardinal) in
// chunks of C rows, four jobs (T2 groups) per chunk as in k_stage_x_tc.  The
// digits of a job are computed straight from the T2 values in global memory
// into one of two digit tiles, so those of job j + 1 are built while the MMAs
// of job j run (the tile waits only for the MMAs of job j - 1).  Lane 0 of warp c issues
// the MMAs of chunk row c: for every K step and A digit i, one M = 128,
// N = 16 (7 - i), K = 16 MMA (see above).
template <int P, int DIM>
__global__ void __launch_bounds__(kTcThreads, 1)
k_stage_x_tc64(Geo g, Tables T, Box b, int i0_lo, int i0_hi, const double* scratch, double* ell, int64_t N)
{
    using Sh = Tc64Shape<P>;
    constexpr int Q = Sh::Q, W = Sh::W, TT = Sh::TT, KW = Sh::KW, C = Sh::C, ROWS = Sh::ROWS;
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    unsigned char* sA = tc_smem;                                         // [tile 2][digit 7][line group 16][ROWS][16 B]
    unsigned char* sB = tc_smem + 2 * Sh::A_BUF;                         // [group 4][digit x 16 + n: 14 groups of 8][K block][128 B]
    float* sScale = reinterpret_cast<float*>(sB + Sh::B_BYTES);          // [group 4][line 128]
    int* sEl = reinterpret_cast<int*>(sScale + 4 * kTcLines);            // [line 128] exponent of the line scale
    int* sEb = sEl + kTcLines;                                           // [16] exponent of the column scale
    uint64_t* bars = reinterpret_cast<uint64_t*>(sEb + kTcN);            // [0..1] digit tile consumed, [2] drain
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    const int64_t G0 = (int64_t)b.E[0] * Q;
    const int64_t P3 = (DIM == 3) ? (int64_t)b.R[2] * W : 1;
    const int64_t P2 = (int64_t)b.R[1] * W;
    const int64_t total = P3 * P2;
    const int64_t line0 = (int64_t)blockIdx.x * kTcLines;
    const float2* T2 = reinterpret_cast<const float2*>(scratch + b.t2_off);
    const int64_t gs = total * G0;
    const int* ex = reinterpret_cast<const int*>(scratch + b.ex_off);
    const int nchunks = (i0_hi - i0_lo) / C + 1;
    const int jobs = 4 * nchunks;

    // line scales: alpha = v 2^(sigma_g - e_line - 1), e_line the recorded largest shifted exponent
    int sig[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) sig[k] = T.gshift[k];
    if (tid < kTcLines) {
        const int64_t line = line0 + tid;
        const int m = (line < total) ? ex[line] : 0;
        const int el = m > 0 ? m - kTcExpOffset - 127 : 0;      // unbiased exponent of the shifted line maximum
        sEl[tid] = el + 1;
#pragma unroll
        for (int k = 0; k < 4; ++k) sScale[k * kTcLines + tid] = m > 0 ? pow2f(sig[k] - el - 1) : 0.f;
    }
    // B: per offset column n the largest exponent of X_g 2^-sigma_g over groups and Gauss points, then
    // six digits of X_g 2^-sigma_g 2^-(e_n + 1), K-major [16 offsets x KW points] per group and digit
    const double* Xc = T.X[0] + (int64_t)(2 * P) * W * TT * 4;
    if (tid < kTcN) sEb[tid] = -100000;
    __syncthreads();
    for (int idx = tid; idx < 4 * W * TT; idx += kTcThreads) {
        const int gq = idx / (W * TT), n = (idx / TT) % W, k = idx % TT;
        const double x = Xc[((int64_t)n * TT + k) * 4 + (3 - gq)];
        if (x != 0.0) atomicMax(&sEb[n], ilogb(x) - sig[gq]);
    }
    __syncthreads();
    for (int idx = tid; idx < 4 * kTcN * KW; idx += kTcThreads) {
        const int gq = idx / (kTcN * KW), n = (idx / KW) % kTcN, k = idx % KW;
        double r = 0.0;
        if (n < W && k < TT && sEb[n] > -100000)
            r = ldexp(Xc[((int64_t)n * TT + k) * 4 + (3 - gq)], -sig[gq] - sEb[n] - 1);
        __nv_bfloat16* base = reinterpret_cast<__nv_bfloat16*>(sB + (size_t)gq * Sh::B_GROUP);
#pragma unroll
        for (int i = 0; i < kDigits; ++i) {
            const double q = rint(ldexp(r, 7 + 8 * i)) * ldexp(1.0, -7 - 8 * i);
            r -= q;
            const int row = i * kTcN + n;             // digit i of offset n: B row 16 i + n
            base[((row >> 3) * (KW / 8) + (k >> 3)) * 64 + (row & 7) * 8 + (k & 7)] = __double2bfloat16(q);
        }
    }
    if (tid == 0) {
        tc::bar_init(&bars[0], kTcThreads / 32);
        tc::bar_init(&bars[1], kTcThreads / 32);
        tc::bar_init(&bars[2], kTcThreads / 32);
        tc::fence_bar_init();
    }
    if (warp == 0) tc::tmem_alloc(tmem_slot, Sh::TMEM_COLS);
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    // the epilogue's output line for this thread (warp w: tensor-memory lanes 32 (w % 4) ..)
    const int q4 = warp & 3, quarter = warp >> 2;
    const int64_t my_line = line0 + q4 * 32 + lane;
    int64_t rowbase = 0;
    int slot0 = 0;
    if (my_line < total) {
        const int64_t pair3 = my_line / P2, pair2 = my_line - pair3 * P2;
        const int i1 = b.rlo[1] + (int)(pair2 / W), d1 = (int)(pair2 % W);
        const int i2 = (DIM == 3) ? b.rlo[2] + (int)(pair3 / W) : 0;
        const int d2 = (DIM == 3) ? (int)(pair3 % W) : 0;
        rowbase = (int64_t)g.m[0] * (i1 + (int64_t)g.m[1] * i2);
        slot0 = W * (d1 + W * d2);
    }
    const int my_el = sEl[q4 * 32 + lane];

    const uint32_t sA_addr = tc::smem_addr(sA), sB_addr = tc::smem_addr(sB);
    bool ok = true;
    int done_chunks = 0;
    for (int j = 0; j < jobs; ++j) {
        const int k = j >> 2, gq = j & 3, buf = j & 1;
        const int c0 = i0_lo + k * C, nc = min(C, i0_hi - c0 + 1);
        // digit tile buf was last read by the MMAs of job j - 2
        // (one warp polls the mbarrier; the others wait at the block barrier without taking issue slots)
        const bool wok = (j >= 2 && warp == 0) ? tc::bar_wait(&bars[buf], (uint32_t)(((j >> 1) - 1) & 1), kTcWaitIter) : true;
        ok = __syncthreads_and(wok) != 0;
        if (!ok) break;
        // digits of the job's T2 values (zero beyond the box), 8 lines x 1 Gauss point per item
        const int64_t row0 = (int64_t)(c0 - P - b.elo[0]) * Q;
        const float2* src = T2 + (int64_t)gq * gs;
        unsigned char* tile = sA + (size_t)buf * Sh::A_BUF;
        for (int item = tid; item < 16 * ROWS; item += kTcThreads) {
            const int lg = item / ROWS, r = item - lg * ROWS;
            const int64_t gp = row0 + r;
            float2 vv[8];
#pragma unroll
            for (int l = 0; l < 8; ++l) {
                const int64_t line = line0 + lg * 8 + l;
                vv[l] = (line < total && gp < G0) ? src[line * G0 + gp] : make_float2(0.f, 0.f);
            }
            uint32_t w[kDigits][4];
#pragma unroll
            for (int l = 0; l < 8; l += 2) {
                float qa[kDigits], qb[kDigits];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int line = lg * 8 + l + u;
                    const float2 v = vv[l + u];
                    const float sc = sScale[gq * kTcLines + line];
                    float rh = __fmul_rn(v.x, sc), rl = __fmul_rn(v.y, sc);
#pragma unroll
                    for (int i = 0; i < kDigits; ++i) {
                        const float up = __int_as_float((127 + 7 + 8 * i) << 23), dn = __int_as_float((127 - 7 - 8 * i) << 23);
                        const float q = __fmul_rn(rintf(__fmul_rn(__fadd_rn(rh, rl), up)), dn);
                        rh = __fsub_rn(rh, q);
                        (u ? qb : qa)[i] = q;
                    }
                }
#pragma unroll
                for (int i = 0; i < kDigits; ++i) w[i][l / 2] = pack2(__float2bfloat16_rn(qa[i]), __float2bfloat16_rn(qb[i]));
            }
            const size_t off = ((size_t)lg * ROWS + r) * 16;
#pragma unroll
            for (int i = 0; i < kDigits; ++i)
                *reinterpret_cast<uint4*>(tile + (size_t)i * Sh::A_SLICE + off) = make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]);
        }
        tc::fence_async_smem();
        __syncthreads();                              // digit tile complete
        if (lane == 0) {
            tc::fence_after_sync();
            const uint64_t a0 = tc::sdesc(sA_addr + (uint32_t)(buf * Sh::A_BUF), 128, ROWS * 16);
            const uint64_t b0 = tc::sdesc(sB_addr + (uint32_t)(gq * Sh::B_GROUP), 128, (KW / 8) * 128);
            for (int c = warp; c < nc; c += kTcThreads / 32) {
#pragma unroll
                for (int ks = 0; ks < Sh::KSTEPS; ++ks) {
                    const uint64_t arow = (uint64_t)(c * Q + ks * 16);
#pragma unroll
                    for (int i = 0; i < kDigits; ++i) {
                        const uint32_t idesc = tc::idesc_bf16_f32(kTcLines, kTcN * (kDigits - i), 1, 0);
                        const uint64_t ad = a0 + (uint64_t)(i * Sh::A_SLICE / 16) + arow;
                        const uint64_t bd = b0 + (uint64_t)(ks * 256 / 16);
                        // the first MMA of the row in the chunk (digit 0, all seven blocks) starts them
                        tc::mma_bf16(tmem + (uint32_t)(c * Sh::NB + i * kTcN), ad, bd, idesc, (gq | ks | i) ? 1u : 0u);
                    }
                }
            }
            tc::commit(&bars[buf]);
        }
        if (gq == 3) {
            // rows of the chunk (once the MMAs of this job, and so of all the chunk's jobs, are done): the
            // level blocks added in double-float, scaled back, rounded to double
            ok = __syncthreads_and(warp == 0 ? tc::bar_wait(&bars[buf], (uint32_t)((j >> 1) & 1), kTcWaitIter) : true) != 0;
            if (!ok) break;
            tc::fence_after_sync();
            for (int c = quarter; c < nc; c += kTcThreads / 128) {
                // level blocks from the smallest up, each added to the row's double-float sums
                float sh[W], sl[W];
#pragma unroll
                for (int dd = 0; dd < W; ++dd) { sh[dd] = 0.f; sl[dd] = 0.f; }
#pragma unroll 1
                for (int a = kDigits - 1; a >= 0; --a) {
                    float v[16];
                    tc::tmem_ld16(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(c * Sh::NB + a * kTcN), v);
#pragma unroll
                    for (int dd = 0; dd < W; ++dd) {
                        const float t = __fadd_rn(sh[dd], v[dd]);
                        const float z = __fsub_rn(t, sh[dd]);
                        sl[dd] = __fadd_rn(sl[dd], __fadd_rn(__fsub_rn(sh[dd], __fsub_rn(t, z)), __fsub_rn(v[dd], z)));
                        sh[dd] = t;
                    }
                }
                if (my_line < total) {
                    const int64_t row = c0 + c + rowbase;
#pragma unroll
                    for (int dd = 0; dd < W; ++dd) {
                        const int e = my_el + sEb[dd] + 1;
                        double out;
                        if (e > -100 && e < 100) {
                            const float f = pow2f(e);
                            out = df2d_exact(__fmul_rn(sh[dd], f), __fmul_rn(sl[dd], f));
                        } else {
                            out = ldexp((double)sh[dd] + (double)sl[dd], e);
                        }
                        ell[(int64_t)(slot0 + dd) * N + row] = (sEb[dd] > -100000) ? out : 0.0;
                    }
                }
            }
            tc::fence_before_sync();
            __syncthreads();
            done_chunks = k + 1;
        }
    }
    if (!ok) {
        tc::cp_async_wait<0>();
        if (tid == 0) atomicOr(&g_tc_status, 1);
        if (lane == 0) tc::commit(&bars[2]);
        tc::bar_wait(&bars[2], 0u, kTcWaitIter);
        if (quarter == 0 && my_line < total)
            for (int i0 = i0_lo + done_chunks * C; i0 <= i0_hi; ++i0)
                for (int dd = 0; dd < W; ++dd)
                    ell[(int64_t)(slot0 + dd) * N + rowbase + i0] = __longlong_as_double(0x7ff8000000000000LL);
    }
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, Sh::TMEM_COLS);
}

template <int P, int DIM, bool F64>
static cudaError_t stage_x_tc_boxes(const Geo& g, const Tables& T, const BoxSet& bs, const double* scratch, void* ell,
                                    int64_t N, cudaStream_t s, bool* used)
{
    constexpr int W = 2 * P + 1;
    constexpr int SMEM = F64 ? Tc64Shape<P>::SMEM : TcShape<P>::SMEM;
    *used = false;
    const int card_lo = 2 * P, card_hi = g.m[0] - 2 * P - 1;
    if (card_hi < card_lo) return cudaSuccess;
    static bool attr_set = false;        // idempotent; set outside any stream capture
    if (!attr_set) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return cudaSuccess;
        cudaError_t e = F64 ? cudaFuncSetAttribute(k_stage_x_tc64<P, DIM>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM)
                            : cudaFuncSetAttribute(k_stage_x_tc<P, DIM>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    for (int k = 0; k < bs.nb; ++k) {
        const Box& b = bs.box[k];
        const int lo = max(card_lo, b.rlo[0]), hi = min(card_hi, b.rlo[0] + b.R[0] - 1);
        if (hi < lo) continue;
        if (F64 && b.ex_off < 0) return cudaErrorInvalidValue;
        const int64_t lines = ((DIM == 3) ? (int64_t)b.R[2] * W : 1) * b.R[1] * W;
        const int64_t grid = (lines + kTcLines - 1) / kTcLines;
        if (grid > 0x7fffffffLL) return cudaErrorInvalidValue;
        launch_begin(K_STAGE_X_TC, s);
        if constexpr (F64)
            k_stage_x_tc64<P, DIM><<<(unsigned)grid, kTcThreads, SMEM, s>>>(g, T, b, lo, hi, scratch, (double*)ell, N);
        else
            k_stage_x_tc<P, DIM><<<(unsigned)grid, kTcThreads, SMEM, s>>>(g, T, b, lo, hi, scratch, (float*)ell, N);
        launch_end(K_STAGE_X_TC, s);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    *used = true;
    return cudaSuccess;
}

template <bool F64>
static cudaError_t stage_x_tc_dispatch(const Geo& g, const Tables& T, const BoxSet& bs, const double* scratch,
                                       void* ell, int64_t N, cudaStream_t s, bool* used)
{
    switch (g.p * 4 + g.dim) {
    case 2 * 4 + 2: return stage_x_tc_boxes<2, 2, F64>(g, T, bs, scratch, ell, N, s, used);
    case 2 * 4 + 3: return stage_x_tc_boxes<2, 3, F64>(g, T, bs, scratch, ell, N, s, used);
    case 3 * 4 + 2: return stage_x_tc_boxes<3, 2, F64>(g, T, bs, scratch, ell, N, s, used);
    case 3 * 4 + 3: return stage_x_tc_boxes<3, 3, F64>(g, T, bs, scratch, ell, N, s, used);
    case 4 * 4 + 2: return stage_x_tc_boxes<4, 2, F64>(g, T, bs, scratch, ell, N, s, used);
    case 4 * 4 + 3: return stage_x_tc_boxes<4, 3, F64>(g, T, bs, scratch, ell, N, s, used);
    case 5 * 4 + 2: return stage_x_tc_boxes<5, 2, F64>(g, T, bs, scratch, ell, N, s, used);
    case 5 * 4 + 3: return stage_x_tc_boxes<5, 3, F64>(g, T, bs, scratch, ell, N, s, used);
    default: return cudaSuccess;
    }
}

// Tensor-core stage X for the cardinal rows of every explicit box (FP32 values
// with T.tc, FP64 values with T.tc64; degrees 2..5); *used tells whether it ran
// (the CUDA-core stage X then skips those rows).
cudaError_t launch_stage_x_tc(const Geo& g, const Tables& T, const BoxSet& bs, const double* scratch, void* ell,
                              int f64, int64_t N, cudaStream_t s, bool* used)
{
    *used = false;
    return f64 ? stage_x_tc_dispatch<true>(g, T, bs, scratch, ell, N, s, used)
               : stage_x_tc_dispatch<false>(g, T, bs, scratch, ell, N, s, used);
}

}  // namespace iga
