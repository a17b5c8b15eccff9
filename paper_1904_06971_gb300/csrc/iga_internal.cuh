// Internal declarations of libiga (CUDA, sm_103a).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "iga.h"

namespace iga {

constexpr int kMaxP = 5;          // degrees 1..5 are instantiated
constexpr int kMaxQ = 7;          // interpolation degree 0..7
constexpr int kBlock = 256;       // threads per block of the item-parallel kernels
constexpr int kLinesX = 2;        // output lines per thread in quadrature stage X
constexpr int kTcExpOffset = 1000;    // per-line T2 exponents are stored as biased exponent + shift + this (0: all zero)

// Geometry map + diffusion coefficient + mesh; passed by value to kernels.
struct Geo {
    int dim, p;
    int n_el[3], m[3];
    int map_kind;
    double amp;
    double aff[12];
    int kappa_kind, kappa_deg;
    double ka, kb;
    double poly[64];
    int knc[3];               // IGA_KAPPA_BSPLINE3: control values per direction
    const double* kctrl;      // IGA_KAPPA_BSPLINE3: control values (device)
    const float2* kctrl_df;   // IGA_KAPPA_BSPLINE3: the same as double-float pairs (scratch), or null
    int kctrl_split;          // the assembly provides kctrl_df (set before prepare_coef_df)
    // double-float copies (hi, lo) of amp, ka, kb for the double-float coefficient path
    float amp_df[2], ka_df[2], kb_df[2];
    int coef_df;              // evaluate the coefficient tensor in double-float arithmetic
    int form;                 // kFormStiffness or kFormMass
};

// Bilinear forms: the diffusion stiffness (Sec. 3.2) and the mass form of Sec. 8.
enum Form { kFormStiffness = 0, kFormMass = 1 };

// A rectangular block of rows whose full stencil rows are computed by the
// sum-factorised quadrature, with the Gauss points it needs.
struct Box {
    int rlo[3], R[3];         // row index range per direction
    int elo[3], E[3];         // element range per direction (covers the rows' supports)
    int out_kind;             // 0: write rows into the ELL values; 1: into the FP64 sample table
    int64_t sample_id;        // column of the sample table (out_kind 1; the box is one row)
    int64_t c_off;            // offset (doubles) of the box's coefficient fields in scratch
    int64_t t1_off, t2_off;   // offsets (doubles) of the stage intermediates
    int64_t blk[4];           // first block of this box in the K2 / Z / Y / X launches
    int64_t ex_off;           // offset (doubles) of the per-line exponents of T2 (tensor-core FP64 stage X), or -1
    // The stiffness matrix is symmetric (A_ij = A_ji).  sym = +1: the stages compute only the
    // upper offsets of the box's rows (colexicographic slot >= the centre: delta_n > 0, or
    // delta_n = 0 and the next component > 0, ...), -1: only the lower ones (slot <= the centre),
    // and a mirror pass copies the rest from the partner rows (which must be rows of the same
    // kind); 0: every offset.
    int sym;
};

constexpr int kMaxBoxes = 7;
constexpr int kMaxV = 2 * kMaxP + 1;      // offset components delta_d = -p..p

// The sample indices of one direction, in increasing order: a run of n_lo
// consecutive indices from c0, n_mid lattice points c0 + (j_first + k) M, and a
// run of n_hi consecutive indices from hi0 (n = n_lo + n_mid + n_hi).
//   common domain Omega~ = [k0, k1]: no low run, the lattice k0 + jM <= k1, and k1
//     as a one-index high run when the lattice misses it (Sec. 6);
//   per-offset domains: the p + 1 first and last cardinal indices as the runs and
//     the lattice p + jM between them (the ends of every Omega~_delta are samples).
struct SampleAxis {
    int c0, M, n_lo, j_first, n_mid, hi0, n_hi, n;
};
__host__ __device__ __forceinline__ int axis_sample(const SampleAxis& a, int k)
{
    if (k < a.n_lo) return a.c0 + k;
    k -= a.n_lo;
    if (k < a.n_mid) return a.c0 + (a.j_first + k) * a.M;
    return a.hi0 + (k - a.n_mid);
}

// The boxes of one assembly: a few explicit boxes (the whole patch, or the
// frame slabs) and an implicit batch of one-row boxes at the sample rows
// s_d = axis_sample(ax_d, a_d), a_d = 0..n_d-1 (sample id a_0 + n_0 (a_1 + n_1 a_2)).
struct BoxSet {
    int nb;
    Box box[kMaxBoxes];
    int64_t n_samples;
    SampleAxis ax[3];
    int64_t s_c_off, s_t1_off, s_t2_off;      // scratch offsets of sample box 0
    int64_t s_c_len, s_t1_len, s_t2_len;      // scratch per sample box
    int64_t blk_s[4];                         // first block of the batch in launch k
    int64_t bper_s[4];                        // blocks per sample box in launch k
};

// Box owning block `block` of launch `stage`.  Every thread of a block gets the same box.
__device__ __forceinline__ void get_box(const BoxSet& bs, int dim, int p, int stage, int64_t block, Box& b)
{
    if (bs.n_samples > 0 && block >= bs.blk_s[stage]) {
        const int64_t sid = (block - bs.blk_s[stage]) / bs.bper_s[stage];
        int64_t rem = sid;
        for (int d = 0; d < 3; ++d) {
            int s = 0;
            if (d < dim) {
                const int a = (int)(rem % bs.ax[d].n);
                rem /= bs.ax[d].n;
                s = axis_sample(bs.ax[d], a);
            }
            b.rlo[d] = s;
            b.R[d] = 1;
            b.elo[d] = (d < dim) ? s - p : 0;
            b.E[d] = (d < dim) ? p + 1 : 1;
        }
        b.out_kind = 1;
        b.ex_off = -1;
        b.sym = 0;
        b.sample_id = sid;
        b.c_off = bs.s_c_off + sid * bs.s_c_len;
        b.t1_off = bs.s_t1_off + sid * bs.s_t1_len;
        b.t2_off = bs.s_t2_off + sid * bs.s_t2_len;
        for (int k = 0; k < 4; ++k) b.blk[k] = bs.blk_s[k] + sid * bs.bper_s[k];
        return;
    }
    int k = bs.nb - 1;
    while (k > 0 && bs.box[k].blk[stage] > block) --k;
    b = bs.box[k];
}

// Per-direction device tables written by the basis kernels.
struct Tables {
    const double* gx[3];      // [G]  Gauss point coordinates xi
    const double* sx[3];      // [2G] sin(pi xi), then sin(2 pi xi)
    const double* cx[3];      // [2G] cos(pi xi), then cos(2 pi xi)
    const double* X[3];       // [m][2p+1][(p+1)^2][4] pair weights (FP64), see k_tables.cu
    const void* Xs[3];        // the same in the store type of the contraction arithmetic
    const float2* tdf[3];     // [G][4] double-float sin(pi xi), pi cos(pi xi), sin(2 pi xi), cos(2 pi xi)
    int arith;                // contraction arithmetic (arith.cuh: kArithF64 / kArithDF / kArithF32)
    int tc;                   // FP32 arithmetic: stage X of the cardinal rows on the tensor cores (k_quad_tc.cu)
    int tc64;                 // double-float arithmetic: the same with exact BF16 digit products (k_quad_tc.cu)
    const int* gshift;        // tc64: [4] exponent shifts sigma_g balancing the T2 groups (k_quad_tc.cu)
};

enum KernelId {
    K_BASIS = 0, K_PAIRS, K_COEF, K_STAGE_Z, K_STAGE_Y, K_STAGE_X,
    K_SPLINE_SETUP, K_SPLINE_SOLVE, K_SPLINE_PARTIAL, K_FILL, K_SPMV, K_DIAG, K_SOLVE,
    K_ADJ_FIELDS, K_ADJ_POINTS, K_ADJ_INTERP, K_ADJ_SAMPLES, K_ADJ_SCATTER, K_STAGE_X_TC, K_MMS, K_PERSIST, K_MIRROR, K_NUM
};

// Launch bookkeeping (iga_api.cu): counts launches and, when profiling is on,
// brackets the launch with events on its stream.
void launch_begin(int kid, cudaStream_t s);
void launch_end(int kid, cudaStream_t s);

// Sets the calling thread's iga_last_error() message; returns code.
int report_error(int code, const char* msg);

// The argument checks of every assembly entry point (patch, degree, map,
// coefficient) and the Geo they describe; sets iga_last_error() and returns
// its status on failure (iga_api.cu).
int validate_geometry(const iga_patch_t* patch, int p, const iga_map_t* map, const iga_kappa_t* kappa, Geo& g);

// Graph capture support (iga_batch.cu): no profiling events while capturing,
// and replays of a captured graph add its kernel count to the launch counter.
void set_capture(bool on);
void add_launches(int64_t n);
int64_t launch_count();
// Drop every cached batch graph that writes into matrix A (iga_batch.cu).
void batch_forget(iga_matrix_t A);
// One patch through the exact (surrogate = false) or surrogate pipeline on `stream`.
int assemble_patch(const iga_patch_t* patch, int p, const iga_map_t* map, const iga_kappa_t* kappa, bool surrogate,
                   int M, int q, int domains, int dtype, void* stream, iga_matrix_t* out);

// ---- one stiffness assembly split into phases (iga_api.cu), for the persistent batch ----
// job_create plans it (argument checks, boxes, sampling lattice, scratch layout)
// and creates the matrix unless `existing` is given; the caller provides the
// scratch (job_scratch_doubles doubles) and runs pre (tables, coefficient
// field), quad (the stage launches, or a persistent launch over PersistWork
// descriptors), post (interpolation, fill) on a stream.
struct Job;
// Everything the persistent quadrature kernel needs of one patch (k_quad.cu);
// done0 indexes its four completion counters (stage Z halves, Y, X).
struct PersistWork {
    Geo g;
    Tables T;
    BoxSet bs;
    double* scratch;
    void* ell;
    double* samples;
    int64_t N;
    int ell_f32;
    int64_t nb[4];            // blocks of the coefficient, Z (per half), Y and X launches
    int64_t done0;
};
int job_create(const iga_patch_t* patch, int p, const iga_map_t* map, const iga_kappa_t* kappa, bool surrogate, int M,
               int q, int domains, int dtype, iga_matrix_t existing, Job** out);
int64_t job_scratch_doubles(const Job* J);
void job_set_scratch(Job* J, double* scratch);
iga_matrix_t job_matrix(const Job* J);
cudaError_t job_pre(Job* J, cudaStream_t s);
cudaError_t job_quad(Job* J, cudaStream_t s);
cudaError_t job_post(Job* J, cudaStream_t s);
// false when the job's stages must run as their own launches (tensor-core stage X)
bool job_persist_work(const Job* J, PersistWork* w);
int job_dim(const Job* J);
int job_degree(const Job* J);
int job_arith(const Job* J);
void job_destroy(Job* J, bool discard_new_matrix);

// A run of consecutive work items of the persistent kernel: blocks 0..count-1
// of stage `stage` (1, 2: Z halves; 3: Y; 4: X) of patch `work`, items
// first..first+count-1.
struct PersistSeg {
    int stage, work;
    int64_t first, count;
};
// Claim counter and status of one persistent launch; zeroed before it.
struct PersistCtl {
    unsigned long long next;  // next unclaimed item
    int abort;                // set when a wait gave up: the other blocks stop
    int status;               // 1: a wait for another block's item ran out of time
};
// Stages Z, Y, X of every work as one launch of `grid` blocks that claim
// `chunk` consecutive items at a time; an item whose stage needs the previous
// stage of its patch waits (bounded by limit_ns of the GPU's global timer) on
// that stage's completion counter in done (4 per work, zeroed).
cudaError_t launch_persist(int dim, int p, int arith, const PersistWork* works, const PersistSeg* segs, int nseg,
                           int64_t total, int chunk, int grid, PersistCtl* ctl, unsigned* done, long long limit_ns,
                           cudaStream_t s);
// Resident blocks per SM of the persistent kernel (0 when the variant is not built).
int persist_blocks_per_sm(int dim, int p, int arith);

// Contraction arithmetic (arith.cuh kind) chosen for matrices of value type dtype,
// and whether its stage X runs on the tensor cores (FP32 values, IGA_ARITH_BF16X3).
int current_arith(int dtype);
int current_tc(int dtype);

// ---- launchers implemented in the kernel files; all return cudaError_t ----
cudaError_t launch_basis(const Geo& g, double* gx[3], double* sx[3], double* cx[3],
                         double* bv[3], double* bd[3], double* wq[3], float2* tdf[3], cudaStream_t s);

// Fill the double-float copies of the map / coefficient constants and decide
// whether the coefficient tensor can be evaluated in double-float arithmetic
// (sine-product map with |amp| <= 0.07, kappa constant / SIN2D / EXPSIN3D with
// |b| <= 1, or BSPLINE3 when g.kctrl_split says the assembly provides kctrl_df).
void prepare_coef_df(Geo& g, int arith);
// The double-float copy of the B-spline coefficient's control values (n values) for the
// double-float coefficient path (k_tables.cu).
cudaError_t launch_split_ctrl(const double* ctrl, int64_t n, float2* out, cudaStream_t s);
cudaError_t launch_pairs(const Geo& g, double* const bv[3], double* const bd[3],
                         double* const wq[3], double* X[3], void* Xs[3], int arith, cudaStream_t s);
cudaError_t launch_coef(const Geo& g, const Tables& T, const BoxSet& bs, int64_t nblocks,
                        double* scratch, cudaStream_t s);
cudaError_t launch_stages(const Geo& g, const Tables& T, const BoxSet& bs, const int64_t nblocks[4],
                          double* scratch, void* ell, int ell_f32, double* samples, cudaStream_t s);
// Mirror of a symmetric matrix over the rows row_begin .. row_begin + count - 1: dir = +1 fills
// every slot below the centre from the partner's upper slot, values[s][i] = values[S-1-s][i + delta_s];
// dir = -1 fills the slots above the centre from the partner's lower slot (0 where i + delta_s lies
// outside the index range).
cudaError_t launch_mirror(int dim, int p, const int m[3], void* values, int f32, int64_t row_begin,
                          int64_t count, int dir, cudaStream_t s);
// Stage X of the cardinal rows of the explicit boxes on the tensor cores: FP32
// values (BF16 parts, FP32 accumulation) or, with T.tc64, FP64 values (six
// BF16 digits, products accumulated exactly per level); p = 2..5; *used =
// false when it did not run.
// The group shifts sigma_g of the FP64 variant (written to gshift, 4 ints) are
// computed from the cardinal pair weights of direction 0 before stage Y, which
// records each T2 line's largest exponent for it.
cudaError_t launch_tc_group_shift(const Geo& g, const Tables& T, int* gshift, cudaStream_t s);
cudaError_t launch_stage_x_tc(const Geo& g, const Tables& T, const BoxSet& bs, const double* scratch, void* ell,
                              int f64, int64_t N, cudaStream_t s, bool* used);
// The same three stages for the mass form: one scalar field (|det Dphi| at the
// Gauss points) and the value-value pair weights only (k_mass.cu).
cudaError_t launch_mass_stages(const Geo& g, const Tables& T, const BoxSet& bs, const int64_t nblocks[4],
                               double* scratch, void* ell, int ell_f32, double* samples, cudaStream_t s);

// Whether the sample index t of a direction is a sample of the variant with
// domain [k0, k1]: every sample in the domain (all != 0, the common domain),
// else the ends and the lattice points c0 + jM at least M/2 away from both
// ends (per-offset domains; the knot spacing then stays within [M/2, 3M/2]).
__host__ __device__ __forceinline__ bool variant_sample(const SampleAxis& ax, int all, int t, int k0, int k1)
{
    if (t < k0 || t > k1) return false;
    if (all || t == k0 || t == k1) return true;
    if ((t - ax.c0) % ax.M) return false;
    return 2 * (t - k0) >= ax.M && 2 * (k1 - t) >= ax.M;
}

// Interpolation plan.  Every offset delta interpolates, in each direction d,
// over the domain [k0, k0 + L - 1] of its component delta_d (variant v = delta_d + p)
// through ns of the direction's samples (variant_sample).  With the common
// domain Omega~ all variants coincide; with per-offset domains they are the
// Omega~_delta of Sec. 3.2.  A variant with L = 0 has no domain.
constexpr int kMaxSamplesPerDir = 2048;
struct SplinePlan {
    int dim, q, S, c, nv;     // nv = 2p + 1 variants per direction
    int first;                // first interpolated slot: c + 1 (kernel-preserving), c (symmetric, diagonal included)
    int all;                  // every variant uses every sample (common domain)
    int64_t n_samples;        // prod nu
    SampleAxis ax[3];
    int nu[3];                // samples per direction (= ax[d].n)
    int r0[3], r1[3];         // rows with interpolated entries: r0 <= i_d <= r1 in every direction
    int k0[3][kMaxV], L[3][kMaxV], ns[3][kMaxV], qe[3][kMaxV];
    int Lmax[3];              // max over variants of L
};
// K4: collocation LU per direction and variant, coefficient solves in place in
// the upper slots of the sample table, evaluation tables and the partially
// evaluated field.
struct SplineBufs {
    int* pos[3][kMaxV];       // [ns] sample positions (axis_sample index) of the variant
    int* inv[3][kMaxV];       // [nu] index into pos of each sample position, or -1
    double* lu[3][kMaxV];     // [ns][ns] LU factors (unit lower L below the diagonal)
    int* band;                // [3][kMaxV][2] lower / upper bandwidth of the factors
    int* espan[3][kMaxV];     // [L] first nonzero basis index (into pos) at domain index k0 + k
    double* eval[3][kMaxV];   // [L][q+1] its values
    float2* eval0[kMaxV];     // direction 0 values again, double-float pairs, transposed [q+1][L]
    float2* partial;          // double-float; 3-D [S_up][Lmax2][Lmax1][nu0]; 2-D [S_up][Lmax1][nu0]
    double* mid;              // 3-D: direction-2 partial sums [S_up][Lmax2][nu1][nu0]
};
cudaError_t launch_spline(const Geo& g, const SplinePlan& sp, double* samples /* [S][n_samples] */,
                          const SplineBufs& sb, cudaStream_t s);
cudaError_t launch_fill(const Geo& g, const SplinePlan& sp, int empty_box, const SplineBufs& sb,
                        void* ell, int ell_f32, cudaStream_t s);
cudaError_t launch_spmv(int dim, int p, const int m[3], const void* values, int f32,
                        const void* x, void* y, cudaStream_t s);
// K4 part 1 alone: knots, collocation LU and evaluation tables of every variant.
cudaError_t launch_spline_setup(const SplinePlan& sp, const SplineBufs& sb, cudaStream_t s);

// ---- manufactured solution u = prod sin(k pi x_d): load a(u, B_i) and energy a(u, u) (k_tables.cu) ----
struct MmsArgs {
    int freq;                 // k
    const double* gx[3];      // [G] Gauss point coordinates
    const double* wq[3];      // [G] weights (times h)
    const double* bv[3];      // [G][p+1] values of the active basis functions
    const double* bd[3];      // [G][p+1] their derivatives
    double* V;                // [dim][points] w kappa |det J| J^{-1} grad u
    double* E;                // [points] w kappa |det J| |grad u|^2
};
// partial: scratch of 2 * npart doubles, npart >= points / (8 * kBlock) + 1
cudaError_t launch_manufactured(const Geo& g, const MmsArgs& A, double* F, double* energy, double* partial,
                                int64_t npart, cudaStream_t s);

// ---- adjoint with respect to B-spline control values of kappa (k_adjoint.cu) ----
struct AdjTables {
    const double* gx[3];      // [G] Gauss point coordinates
    const double* sx[3];      // [G] sin(pi xi) (first G entries of the basis tables)
    const double* cx[3];      // [G] cos(pi xi)
    const double* wq[3];      // [G] weights (times h)
    const double* bv[3];      // [G][p+1] values of the active basis functions
    const double* bd[3];      // [G][p+1] their derivatives
};
constexpr int kMaxAdjTerms = 3;
// s(g) = w_g sum_t sign_t grad u_{a_t}^T G grad u_{b_t}; Wa/Wb are direction-1 partial sums (pass 1)
struct AdjTerms {
    int n;
    double sign[kMaxAdjTerms];
    const double* Wa[kMaxAdjTerms];
    const double* Wb[kMaxAdjTerms];
    int64_t tot1;             // entries per component of a pass-1 array
};
cudaError_t launch_adj_vectors(const Geo& g, const SplinePlan& sp, const double* ybar, const double* x, double* out,
                               cudaStream_t s);
cudaError_t launch_adj_grad_field(const Geo& g, const AdjTables& T, const double* v, double* W0, double* W1,
                                  cudaStream_t s);
cudaError_t launch_adj_points(const Geo& g, const AdjTables& T, const AdjTerms& terms, double* spt, cudaStream_t s);
cudaError_t launch_adj_interp(const Geo& g, const SplinePlan& sp, const SplineBufs& sb, const double* ybar,
                              const double* x, double* C0, double* C1, double* table, cudaStream_t s);
cudaError_t launch_adj_samples(const Geo& g, const AdjTables& T, const SplinePlan& sp, const double* phibar,
                               double* spt, cudaStream_t s);
cudaError_t launch_adj_scatter(const Geo& g, const AdjTables& T, const double* spt, double* grad, cudaStream_t s);

// Scratch sizes (doubles) of a box for the quadrature stages.
inline int64_t box_coef_len(int dim, int p, const Box& b) {
    int Q = p + 1;
    int64_t n = (dim == 3 ? 6 : 3);
    for (int d = 0; d < dim; ++d) n *= (int64_t)b.E[d] * Q;
    return n;
}
inline int64_t box_t1_len(int dim, int p, const Box& b) {
    if (dim != 3) return 0;
    int Q = p + 1, W = 2 * p + 1;
    return (int64_t)8 * b.R[2] * W * ((int64_t)b.E[1] * Q) * ((int64_t)b.E[0] * Q);
}
inline int64_t box_t2_len(int dim, int p, const Box& b) {
    int Q = p + 1, W = 2 * p + 1;
    int64_t pairs3 = (dim == 3) ? (int64_t)b.R[2] * W : 1;
    return (int64_t)4 * pairs3 * ((int64_t)b.R[1] * W) * ((int64_t)b.E[0] * Q);
}
// items of each launch for one box
inline int64_t box_items(int dim, int p, const Box& b, int stage) {
    int Q = p + 1, W = 2 * p + 1;
    int64_t G0 = (int64_t)b.E[0] * Q, G1 = (int64_t)b.E[1] * Q, G2 = (dim == 3) ? (int64_t)b.E[2] * Q : 1;
    int64_t P3 = (dim == 3) ? (int64_t)b.R[2] * W : 1;
    switch (stage) {
        case 0: return G0 * G1 * G2;                         // coefficient points
        case 1: return (dim == 3) ? (int64_t)b.R[2] * G1 * G0 : 0;  // stage Z
        case 2: return P3 * b.R[1] * G0;                     // stage Y
        default: return P3 * (((int64_t)b.R[1] * W + kLinesX - 1) / kLinesX) * b.R[0]; // stage X
    }
}

}  // namespace iga
