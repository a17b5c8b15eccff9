/*
 * iga.h -- C ABI of libiga: GPU (sm_103a) assembly of exact and surrogate
 * stiffness (and mass) matrices for isogeometric analysis on one mapped
 * tensor-product B-spline patch, and the stencil SpMV with the result.
 *
 * The operator is the variable-coefficient diffusion form pulled back to the
 * parametric domain (0,1)^n (Drzisga, Keith & Wohlmuth, "The surrogate matrix
 * methodology: low-cost assembly for isogeometric analysis", Sec. 3.2,
 * eq. BilinearFormPoissonTensor):
 *
 *   A_ij = int grad B_i^T K grad B_j,  K = kappa(phi) |det Dphi| Dphi^{-1} Dphi^{-T},
 *
 * with the open uniform B-spline basis of Sec. 2.2 (degree p, n_el elements
 * and m = n_el + p functions per direction, colexicographic global numbering
 * i = i_0 + m_0 (i_1 + m_1 i_2), 0-based) and (p+1)-point Gauss-Legendre
 * quadrature on every element.
 *
 * Matrix storage ("stencil-ELL", index free): values[s * N + i] holds
 * A_{i, i + delta_s} where the slot s = sum_d (delta_d + p)(2p+1)^d enumerates
 * the (2p+1)^n offsets delta in {-p..p}^n colexicographically (Sec. 3.2: the
 * set D of relevant translations).  Slots whose column leaves the index
 * range hold 0.  The centre slot (S-1)/2 is the diagonal; slot s > (S-1)/2
 * means j > i, and slot S-1-s is the transposed offset.
 *
 * Conventions for every call:
 *   - return value: IGA_OK (0) or a negative IGA_E* code; iga_last_error()
 *     gives a message for the calling thread.  No call traps the device or
 *     throws across the ABI.
 *   - stream: a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Work is enqueued on it; results are valid once it has been
 *     synchronised.  Host-side argument checks happen before anything is
 *     enqueued.
 *   - device memory: the library allocates the matrix values and its scratch
 *     from a library-owned stream-ordered memory pool on the current device;
 *     the pool keeps released blocks for reuse.  Caller pointers (x, y) are
 *     never freed by the library.
 *   - the matrix is the full pure-Neumann matrix; Dirichlet elimination is
 *     the solver's business (Sec. 6, Remark with eq. BlockSystem).
 */
#ifndef IGA_H
#define IGA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define IGA_OK            0
#define IGA_EINVAL       (-1)   /* bad argument (null pointer, size, kind) */
#define IGA_ENOMEM       (-2)   /* device allocation failed */
#define IGA_ECUDA        (-3)   /* a CUDA runtime call or launch failed */
#define IGA_EUNSUPPORTED (-4)   /* valid request outside what is built (p, n, q range) */
#define IGA_ETIMEOUT     (-5)   /* a bounded device wait gave up (persistent batch kernel); the context stays usable */

/* storage type of matrix values and of the SpMV vectors */
#define IGA_F64 0
#define IGA_F32 1

/* geometry maps phi: (0,1)^n -> R^n */
#define IGA_MAP_IDENTITY 0      /* x = xi */
#define IGA_MAP_AFFINE   1      /* x = A xi + b; affine[0..8] = A row-major (3x3; 2-D uses the top-left 2x2), affine[9..11] = b */
#define IGA_MAP_SINPROD  2      /* x_a = xi_a + amp * prod_j sin(pi xi_j) */

/* diffusion coefficients kappa(x), evaluated at the physical point x = phi(xi) */
#define IGA_KAPPA_CONST    0    /* a */
#define IGA_KAPPA_SIN2D    1    /* a + b sin(2 pi x) sin(2 pi y) */
#define IGA_KAPPA_EXPSIN3D 2    /* exp(b sin(2 pi x) cos(2 pi y) sin(2 pi z)) */
#define IGA_KAPPA_POLY     3    /* sum_{a,b,c <= deg} poly[a + (deg+1)(b + (deg+1)c)] x^a y^b z^c, deg <= 3 */
#define IGA_KAPPA_BSPLINE3 4    /* sum ctrl[a + n0 (b + n1 c)] N_a(x) N_b(y) N_c(z): cubic B-splines with open
                                   uniform knots on [0, 1], nctrl_d - 3 elements per direction; the physical
                                   point is clamped onto the unit cube */

/*
 * Arithmetic of the sum-factorised quadrature contractions (process-wide,
 * chosen per value dtype).  The basis tables and pair weights are FP64 in
 * every mode.  The coefficient tensor (and the mass form's |det Dphi|) is FP64
 * too, except on the sine-product map with |amp| <= 0.07 and a constant,
 * SIN2D or EXPSIN3D (|b| <= 1) kappa: there DF64 mode evaluates it in
 * double-float arithmetic and FP32 mode in FP32.
 *   IGA_ARITH_FP64: native FP64 FMAs.
 *   IGA_ARITH_DF64: double-float arithmetic on the FP32 units -- each value is
 *     an unevaluated sum of two floats (about 48 significand bits), products
 *     are formed exactly with an FMA and sums with an error-free two-sum.
 *     GB300 runs FP32 about 64x faster than FP64, so this is the default for
 *     IGA_F64 values; its results agree with FP64 to ~1e-14 relative to the
 *     largest entry.
 *   IGA_ARITH_FP32: FP32 FMAs (only for IGA_F32 values; the default there).
 *   IGA_ARITH_BF16X3: IGA_ARITH_FP32, except that the last contraction (stage X,
 *     direction 0) of the rows whose stencil stays among cardinal B-splines runs
 *     on the tensor cores: each FP32 operand split into three BF16 parts, the six
 *     partial products of order <= 2 accumulated in FP32 (FP32-level accuracy,
 *     Sec. 6 sum factorisation).  Only for IGA_F32 values, degrees 2..5.
 *   IGA_ARITH_DF64_TC: IGA_ARITH_DF64, except that stage X of those rows runs
 *     on the tensor cores with FP64 accuracy: every operand is scaled per T2
 *     line and per offset column by a power of two and written as six signed
 *     base-256 digits in BF16; the digit products of each level are summed
 *     exactly in FP32 tensor memory (levels 0, 1, 2 apart, 3..5 together,
 *     higher levels dropped, below 2^-48), then added in double-float and
 *     rounded once.  Only for IGA_F64 values, degrees 2..5.
 */
#define IGA_ARITH_FP64 0
#define IGA_ARITH_DF64 1
#define IGA_ARITH_FP32 2
#define IGA_ARITH_BF16X3 3
#define IGA_ARITH_DF64_TC 4

typedef struct {
    int32_t dim;        /* n: 2 or 3 */
    int32_t n_el[3];    /* elements per direction (entries beyond dim ignored); n_el >= p + 1 (m >= 2p+1, Sec. 2.2) */
} iga_patch_t;

typedef struct {
    int32_t kind;       /* IGA_MAP_* */
    double amp;         /* IGA_MAP_SINPROD amplitude */
    double affine[12];  /* IGA_MAP_AFFINE coefficients */
} iga_map_t;

typedef struct {
    int32_t kind;       /* IGA_KAPPA_* */
    int32_t deg;        /* IGA_KAPPA_POLY degree per direction (0..3) */
    double a, b;        /* constants of the closed forms above */
    double poly[64];    /* IGA_KAPPA_POLY coefficients */
    int32_t nctrl[3];   /* IGA_KAPPA_BSPLINE3 control values per direction, 4..64 (entries beyond dim ignored) */
    const double* ctrl; /* IGA_KAPPA_BSPLINE3 control values, DEVICE pointer owned by the caller; read by
                           the kernels the call enqueues, so it must stay valid until they complete */
} iga_kappa_t;

typedef struct iga_matrix* iga_matrix_t;   /* opaque; owns device storage */

/*
 * Exact assembly (Sec. 6: the matrix A every entry of which comes from
 * quadrature; eq. ChangeOfVars).  Every row is computed by sum-factorised
 * Gauss quadrature on the GPU.  A is symmetric (A_ij = A_ji: the bilinear form
 * of Sec. 2 with a symmetric coefficient tensor), so the quadrature computes
 * the upper offsets of every row and the lower ones are copied from the partner
 * rows: values[s][i] equals values[S-1-s][i + delta_s] bit for bit (except with
 * IGA_ARITH_BF16X3 / IGA_ARITH_DF64_TC, whose tensor-core stage computes every
 * offset).
 *   patch, map, kappa: host pointers, read during the call only.
 *   p: degree 1..5.  dtype: IGA_F64 or IGA_F32; the contraction arithmetic is the
 *   one iga_set_arithmetic selects for that dtype (FP64 values: double-float by
 *   default; FP32 values: FP32).
 *   A: in/out.  *A == NULL: a new matrix is created.  *A != NULL: a matrix
 *   from an earlier call with the same patch, p and dtype, whose storage is
 *   reused (its previous values are overwritten); otherwise IGA_EINVAL.
 */
int iga_assemble_exact(const iga_patch_t* patch, int p, const iga_map_t* map,
                       const iga_kappa_t* kappa, int dtype, void* stream,
                       iga_matrix_t* A);

/*
 * Surrogate assembly, eq. DefinitionOfSurrogateMatrixSymmetricKernel
 * (Sec. 5.3) with the sampling of Sec. 6:
 *   - Omega~ (Sec. 4) is the index box [2p, m-2p-1] per direction;
 *   - rows with an index outside it ("frame" rows) are exact;
 *   - samples: every M-th index of the box from its first index, plus its
 *     last index; the stencil values Phi_delta at the sample rows are exact;
 *   - per upper offset delta, a degree-q tensor-product B-spline interpolant
 *     through the samples (not-a-knot knots at the sample indices, odd q, or
 *     at their midpoints, even q; degree lowered to n_s - 1 with fewer than
 *     q + 1 samples) gives A~_ij for i < j with i, j in Omega~;
 *   - A~_ij for i > j in Omega~ is the copy A~_ji; every other off-diagonal
 *     entry is exact; every diagonal entry is minus its row's off-diagonal sum.
 *   M >= 1 (M = 1 reproduces the exact matrix), 0 <= q <= 7.  Other arguments
 *   as for iga_assemble_exact.
 */
int iga_assemble_surrogate(const iga_patch_t* patch, int p, const iga_map_t* map,
                           const iga_kappa_t* kappa, int M, int q, int dtype,
                           void* stream, iga_matrix_t* A);

/*
 * Choice of the interpolation domains of the surrogate.
 *   IGA_DOMAINS_COMMON: every stencil function is interpolated on the common
 *     set Omega~ of Sec. 4 (the index box [2p, m-2p-1]); rows outside it are
 *     exact (iga_assemble_surrogate).
 *   IGA_DOMAINS_PER_OFFSET: each stencil function Phi_delta is interpolated on
 *     its own domain Omega~_delta (Sec. 3.2, and Sec. 4 on reformulating with
 *     one interpolation operator per delta): the indices k with k and k + delta
 *     both cardinal, i.e. in [p, m-p-1] in every direction.  Only entries with a
 *     non-cardinal basis function are exact, so exact rows are the frame of
 *     width p.  Samples per direction: every M-th index from p, and the p + 1
 *     first and last cardinal indices (the ends of every Omega~_delta); each
 *     offset interpolates through the samples inside its own domain.
 */
#define IGA_DOMAINS_COMMON 0
#define IGA_DOMAINS_PER_OFFSET 1

/*
 * Surrogate assembly (eq. DefinitionOfSurrogateMatrixSymmetricKernel) with the
 * interpolation domains chosen by `domains` (IGA_DOMAINS_*): for i < j with
 * x~_i in the domain of delta = x~_j - x~_i, A~_ij = Phi~_delta(x~_i); for i > j
 * the copy A~_ji; every other off-diagonal entry exact; every diagonal entry
 * minus its row's off-diagonal sum.  IGA_DOMAINS_COMMON is iga_assemble_surrogate.
 * An unknown `domains` value returns IGA_EINVAL.  Other arguments as for
 * iga_assemble_surrogate.
 */
int iga_assemble_surrogate_domains(const iga_patch_t* patch, int p, const iga_map_t* map,
                                   const iga_kappa_t* kappa, int M, int q, int domains,
                                   int dtype, void* stream, iga_matrix_t* A);

/*
 * Sampling plan of a surrogate assembly, computed on the host only (no device
 * call; usable without a GPU): the sample rows of Sec. 6 per direction and,
 * per direction and offset component delta_d = -p..p, the interpolation domain
 * and the samples inside it, exactly as iga_assemble_surrogate_domains (and,
 * with IGA_DOMAINS_COMMON, iga_assemble_mass_surrogate) uses them.
 *   patch, p, M, q, domains: as for iga_assemble_surrogate_domains.
 *   cap: capacity per direction of `samples`.
 *   samples: host int32 [3][cap]; direction d's sample indices, increasing, at samples[d * cap].
 *   n_samples: host int32 [3]; the count per direction (1, with sample index 0, beyond dim).
 *   dom_lo, dom_hi, dom_ns, dom_q: host int32 [3][2p+1], or all NULL; entry d (2p+1) + (delta_d + p):
 *     the domain's first and last index (Omega~ = [2p, m-2p-1] for every component with
 *     IGA_DOMAINS_COMMON; Omega~_delta's factor [p + max(0,-delta_d), m-p-1-max(0,delta_d)] with
 *     IGA_DOMAINS_PER_OFFSET; an empty domain has hi = lo - 1 and no sample), the number of samples
 *     in it, and the interpolation degree used (q lowered to that number - 1; 0 for an empty domain).
 *   empty: host int; 1 when the region of interpolated rows has no row (every row exact), and
 *     then nothing else is written.
 * Errors: IGA_EINVAL / IGA_EUNSUPPORTED for arguments the assembly rejects, IGA_EINVAL when a
 * direction has more than cap samples.
 */
int iga_surrogate_plan(const iga_patch_t* patch, int p, int M, int q, int domains, int cap, int32_t* samples,
                       int32_t* n_samples, int32_t* dom_lo, int32_t* dom_hi, int32_t* dom_ns, int32_t* dom_q,
                       int* empty);

/*
 * Mass matrix M_ij = int_Omega B_i B_j dx = int B_i B_j |det Dphi| dxi (Sec. 8,
 * proof of the mass-matrix corollary), by the same (p+1)-point Gauss rule and
 * sum-factorised quadrature as iga_assemble_exact, with |det Dphi| as the
 * only coefficient field.  Same stencil-ELL layout; no kappa.  Other arguments
 * as for iga_assemble_exact (the handle is interchangeable with a stiffness
 * matrix of the same patch, p and dtype).
 */
int iga_assemble_mass(const iga_patch_t* patch, int p, const iga_map_t* map, int dtype, void* stream,
                      iga_matrix_t* A);

/*
 * Surrogate mass matrix, eq. DefinitionOfSurrogateMatrixSymmetric (Sec. 5.2):
 * the mass matrix has no kernel, so no row-sum diagonal.  On the common domain
 * Omega~ = [2p, m-2p-1] (Sec. 4) and the samples of iga_assemble_surrogate,
 * the (S+1)/2 stencil functions of the offsets delta >= 0 (colexicographic,
 * the centre included) are interpolated; for i, j in Omega~, M~_ij is
 * Phi~_delta(x~_i) when i <= j (the diagonal included) and the copy M~_ji when
 * i > j; every other entry is exact.  M = 1 reproduces iga_assemble_mass; for
 * an affine map and q >= dim - 1 the surrogate is exact (mass-matrix corollary
 * of Sec. 8).  Arguments as for iga_assemble_surrogate without kappa.
 */
int iga_assemble_mass_surrogate(const iga_patch_t* patch, int p, const iga_map_t* map, int M, int q, int dtype,
                                void* stream, iga_matrix_t* A);

/*
 * Gradient with respect to the B-spline control values of kappa
 * (IGA_KAPPA_BSPLINE3) of L = ybar^T A x, A the exact matrix (M = 0) or the
 * surrogate with the common domain Omega~ (M >= 1, interpolation degree q), as
 * assembled by iga_assemble_exact / iga_assemble_surrogate.  Every step of the
 * surrogate is linear in kappa (the quadrature of eq. ChangeOfVars, the
 * interpolation of Sec. 4.1, the copy and the diagonal of Sec. 5.3), and
 *   dL/dc_k = sum_g N_k(phi(g)) s(g),
 * s(g) the derivative of L with respect to kappa at Gauss point g (bilinear
 * forms of the exact entries, the transposed interpolation of the interpolated
 * ones).  The gradient with respect to x is A ybar (A is symmetric): use
 * iga_apply.  The basis tables are recomputed by the call; FP64 throughout.
 *   ybar, x: device FP64 [N], colexicographic.  grad: device FP64
 *   [nctrl_0 nctrl_1 (nctrl_2)], overwritten.  kappa->ctrl is read.
 *   Errors: IGA_EINVAL for another kappa kind, null pointers or M < 0.
 */
int iga_kappa_gradient(const iga_patch_t* patch, int p, const iga_map_t* map, const iga_kappa_t* kappa,
                       int M, int q, const double* ybar, const double* x, double* grad, void* stream);

/*
 * Batched assembly (no counterpart in the paper, which assembles one patch;
 * per patch it is the method of Sec. 6 -- quadrature of the exact rows and
 * sample rows, interpolation, fill): many patches of uneven size, degree, map
 * and coefficient as one CUDA graph.  Item k is assembled like
 * iga_assemble_surrogate_domains (M >= 1) or iga_assemble_exact (M = 0) into A[k].
 *   First call with any A[k] == NULL: every matrix is created by an eager
 *   assembly on `stream` (handles returned in A).  Calls with all handles set:
 *   the batch (descriptions, handles, dtype and contraction arithmetic) is
 *   looked up in a graph cache; on a miss an autotuner captures candidate graphs
 *   and keeps the fastest of two timed replays (this first graph call
 *   synchronises); on a hit the cached graph is launched on `stream` as one
 *   graph launch.  Candidates (iga_batch_set_modes restricts them):
 *     branches: every patch's kernel chain on B concurrent branches, B = 1, 2,
 *       4, ..., 32;
 *     persistent: the quadrature stages of all patches of one (dimension,
 *       degree, arithmetic) as ONE persistent kernel over device-side patch
 *       descriptors -- work items are the stage blocks, claimed from a device
 *       counter; an item waits for the previous stage of its patch on a
 *       completion counter, each wait bounded (2 s of the GPU's global timer);
 *       tuned over resident blocks per SM and items per claim.  Not used with
 *       the tensor-core stage X modes.  Its scratch is one device allocation
 *       owned by the cached graph (freed by iga_batch_release or when a matrix
 *       of the batch is destroyed).
 *   Device pointers in the descriptions (IGA_KAPPA_BSPLINE3 control values) are
 *   captured by address.
 *   Errors: IGA_EINVAL for n < 1, null arrays or a bad dtype; item errors as for
 *   the single-patch calls; IGA_ETIMEOUT when a persistent wait gave up during
 *   tuning (replays report it through iga_batch_status).
 */
typedef struct {
    iga_patch_t patch;
    int32_t p;
    iga_map_t map;
    iga_kappa_t kappa;
    int32_t M;          /* >= 1: surrogate with sampling parameter M; 0: exact matrix */
    int32_t q;          /* interpolation degree (surrogate) */
    int32_t domains;    /* IGA_DOMAINS_* (surrogate) */
} iga_batch_item_t;

int iga_assemble_batch(int n, const iga_batch_item_t* items, int dtype, void* stream, iga_matrix_t* A);

/* The calling thread's last iga_assemble_batch: concurrent branches of its graph
 * (0 for the eager first call), kernels per replay, 1 if the graph came from the
 * cache, and the tuned replay time in ms (0 unless a graph was tuned). */
int iga_batch_info(int* branches, int64_t* kernels, int* cached, float* tuned_ms);

/* Destroys every cached batch graph (iga_matrix_destroy already drops the graphs
 * that write into the destroyed matrix). */
int iga_batch_release(void);

/* Restricts the batch autotuner's candidates (process-wide; both allowed by
 * default; at least one must be).  Affects graphs tuned after the call. */
int iga_batch_set_modes(int allow_branches, int allow_persistent);

/* The calling thread's last iga_assemble_batch: 1 if its graph is the
 * persistent kind, with the tuned resident blocks per SM and items per claim. */
int iga_batch_mode(int* persistent, int* blocks_per_sm, int* chunk);

/* Synchronises `stream` and returns IGA_ETIMEOUT if a wait of the calling
 * thread's last persistent batch replay gave up, else IGA_OK. */
int iga_batch_status(void* stream);

/* Self-test of the bounded wait: launches the persistent kernel on one work
 * item whose dependency nothing ever completes; the wait must give up after
 * limit_us microseconds (1..1e7) and the call returns IGA_ETIMEOUT with the
 * device still usable (IGA_OK would mean the wait did not run out). */
int iga_batch_selftest_timeout(long long limit_us, void* stream);

/*
 * y = A x (eq. DiscreteVariationalProblems), stencil SpMV.  x and y are
 * caller-owned DEVICE arrays of N elements of the matrix dtype (double for
 * IGA_F64, float for IGA_F32); x and y must not overlap.
 */
int iga_apply(iga_matrix_t A, const void* x, void* y, void* stream);

/*
 * y = A x with HOST arrays (pinned or pageable): the call copies x to the
 * device, runs the SpMV and copies y back on `stream`, and returns after the
 * stream has been synchronised.  Uses a library-owned device staging buffer.
 */
int iga_apply_host(iga_matrix_t A, const void* x_host, void* y_host, void* stream);

/*
 * Conjugate gradients on the Dirichlet-reduced system A_II u_I = f_I (Sec. 6,
 * Remark with eq. BlockSystem: the dofs of basis functions with an index 0 or
 * m-1 in some direction carry homogeneous Dirichlet values and are
 * eliminated).  f, u: caller-owned DEVICE arrays of N doubles; f's Dirichlet
 * entries are ignored, u returns the solution with zeros on Dirichlet dofs
 * (the start vector is zero).  Stops when ||f_I - A_II u_I|| <= tol ||f_I|| or
 * after maxit CG iterations.  IGA_F64 matrices: CG in FP64.  IGA_F32
 * matrices: iterative refinement -- the residual is computed in FP64 (the
 * FP32 values promoted), an FP32 CG solves for the correction to 1e-4, and
 * the correction is added in FP64.  iters / relres return the total CG
 * iterations and the final relative residual (FP64).  Synchronises `stream`.
 */
int iga_cg(iga_matrix_t A, const double* f, double* u, double tol, int maxit, void* stream,
           int* iters, double* relres);

/* Sizes: N dofs, S slots, structural nonzeros prod_d(m_d(2p+1) - p(p+1)), dtype. Any out pointer may be NULL. */
int iga_matrix_info(iga_matrix_t A, int64_t* N, int32_t* S, int64_t* nnz, int32_t* dtype);

/* Device pointer to the values array [S][N] (owned by A; valid until destroy or re-assembly). */
int iga_matrix_values(iga_matrix_t A, const void** values);

/* Copy all S*N values to dst (host if dst_on_host != 0, else device); synchronises `stream`. */
int iga_matrix_copy_values(iga_matrix_t A, void* dst, int dst_on_host, void* stream);

/* Release A and its device storage (stream-ordered on the stream of its last assembly). NULL is a no-op. */
int iga_matrix_destroy(iga_matrix_t A);

/* Set / query the contraction arithmetic used by later assemblies of dtype
 * values (IGA_F32 accepts all three, IGA_F64 only FP64 and DF64). */
int iga_set_arithmetic(int dtype, int arith);
int iga_get_arithmetic(int dtype);

/*
 * Counters for benchmarking: number of kernels this library launched in the
 * calling process since start (monotone), and per-kernel device time.
 * iga_profile_enable(1) makes every later launch record a pair of CUDA
 * events on its stream; iga_profile_read() synchronises those events and
 * returns, for kernel id k < n, the number of launches and total
 * milliseconds, then clears them.  Names come from iga_kernel_name(k).
 */
int64_t iga_launch_count(void);
int iga_profile_enable(int on);
int iga_profile_read(int n, int64_t* launches, double* ms);
int iga_num_kernels(void);
const char* iga_kernel_name(int k);

/*
 * Load vector and energy of the manufactured solution u(x) = prod_d sin(k pi x_d)
 * (k = freq in 1..1000; the paper's Poisson experiments use k = 1 and k = 20,
 * Sec. 7.3), for the split of a
 * surrogate solution's error into discretisation and consistency parts (the
 * two terms of the a-priori bounds, eq. APrioriBoundH1; rule of thumb: keep the
 * consistency error at or below 5 % of the discretisation error):
 *   F[i]    = a(u, B_i) = int kappa grad u . grad B_i dx   (i = 0..N-1, colexicographic),
 *   *energy = a(u, u)   = int kappa |grad u|^2 dx,
 * both with the assembly's (p+1)-point Gauss rule, pulled back through the map
 * (eq. ChangeOfVars), in FP64.  u vanishes on the boundary of the unit square /
 * cube, so for maps of it onto itself (identity, sine-product) u solves the
 * homogeneous Dirichlet problem whose Galerkin load is F, and for the solution
 * u_h of A_II u_h = F_I: ||u - u_h||_a^2 = a(u, u) - F . u_h.
 *   F, energy: caller-owned DEVICE buffers of N and 1 doubles; the call is
 *   enqueued on the stream and allocates its scratch from the library's pool.
 */
int iga_manufactured_load(const iga_patch_t* patch, int p, const iga_map_t* map, const iga_kappa_t* kappa,
                          int freq, double* F, double* energy, void* stream);

/*
 * Exact assembly that allocates no memory (the paper has no counterpart; this
 * serves callers that may not allocate device memory during a call -- e.g.
 * latency-critical loops where cudaMalloc/cudaFree would synchronise or
 * stall, or applications whose own allocator owns the GPU's memory).
 *   values: caller-owned DEVICE buffer of S * N elements of dtype (double or
 *   float), written with the stencil-ELL layout above; the other arguments
 *   are those of iga_assemble_exact and are checked the same way (every map
 *   and coefficient kind, IGA_KAPPA_BSPLINE3 included: its control values are
 *   the caller's device memory).  Its quadrature computes every offset of
 *   every row (no mirror pass), so its values equal those of iga_assemble_exact
 *   to rounding, not bit for bit in the lower half.
 * Scratch: one file-scope device array of 64 MiB that every GPU which loads
 * this library reserves until the process exits.  A patch whose quadrature
 * scratch exceeds 64 MiB is rejected with IGA_EUNSUPPORTED before any work
 * (e.g. 3-D p = 3 fits up to about 12^3 elements, p = 2 up to 16^3; 2-D p = 2
 * up to several hundred elements per direction).
 * The first call on a device looks up the array's device address (with that
 * device current) and keeps it for the life of the process; make that first
 * call before any stream capture.  The kept address is not valid after
 * cudaDeviceReset() or another teardown of the device's primary context.
 * Every call uses the same array, so calls whose work overlaps on the GPU
 * (other streams, other host threads) race and must be serialised by the
 * caller.  No part of the array needs to start at zero: every word a call
 * reads is written earlier in the same call.
 */
int iga_assemble_exact_noalloc(const iga_patch_t* patch, int p, const iga_map_t* map,
                               const iga_kappa_t* kappa, int dtype, void* values, void* stream);

/* Self-test of the double-float sin / cos / exp used by the coefficient kernel:
 * their maximum errors against CUDA's FP64 sincospi and exp on n points of
 * their domains (|pi y| <= 0.5, |x| <= 1) go to errors[0..2] (sin and cos
 * absolute, exp relative).  Synchronous; allocates a few bytes. */
int iga_selftest_dfmath(int n, double* errors);

/* Thread-local message for the last failing call on this thread ("" if none). */
const char* iga_last_error(void);

/* ABI version (major * 10000 + minor * 100 + patch). */
int iga_version(void);

#ifdef __cplusplus
}
#endif

#endif /* IGA_H */
