// libiga C ABI (include/iga.h): argument checks, planning of the quadrature
// boxes and the sampling lattice, scratch layout, and the launch sequence.
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "arith.cuh"
#include "iga_internal.cuh"

using namespace iga;

struct iga_matrix {
    int dim, p, dtype;
    int n_el[3], m[3];
    int64_t N, nnz;
    int S;
    void* values;             // [S][N], cudaMalloc'd
    size_t bytes;
    int device;
};

namespace {

thread_local std::string t_err;

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    t_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    return fail(e == cudaErrorMemoryAllocation ? IGA_ENOMEM : IGA_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ---- contraction arithmetic per value dtype (process-wide) ----
std::atomic<int> g_arith[2] = {{kArithDF}, {kArithF32}};
std::atomic<int> g_tc_f32{0};          // FP32 values: stage X of the cardinal rows on the tensor cores
std::atomic<int> g_tc_f64{0};          // FP64 values: the same with exact BF16 digit products

// ---- launch counting and optional per-kernel event timing ----
std::atomic<int64_t> g_launches{0};
std::atomic<int> g_profile{0};
std::mutex g_prof_mu;
struct Pending { int kid; cudaEvent_t a, b; };
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_events;
thread_local cudaEvent_t t_begin = nullptr;
thread_local bool t_capture = false;        // inside a graph capture: no profiling events

const char* kNames[K_NUM] = {"basis", "pairs", "coef", "stage_z", "stage_y", "stage_x",
                             "spline_setup", "spline_solve", "spline_partial", "fill", "spmv", "diag", "cg",
                             "adj_fields", "adj_points", "adj_interp", "adj_samples", "adj_scatter", "stage_x_tc",
                             "manufactured", "persist", "mirror"};

cudaEvent_t take_event()
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_events.empty()) {
        cudaEvent_t e = g_events.back();
        g_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// ---- library-owned stream-ordered pool per device (keeps freed blocks) ----
std::mutex g_pool_mu;
cudaMemPool_t g_pools[128] = {};

cudaError_t device_pool(int dev, cudaMemPool_t* out)
{
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    if (!g_pools[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaError_t e = cudaMemPoolCreate(&g_pools[dev], &props);
        if (e != cudaSuccess) { g_pools[dev] = nullptr; return e; }
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(g_pools[dev], cudaMemPoolAttrReleaseThreshold, &thr);
    }
    *out = g_pools[dev];
    return cudaSuccess;
}

int64_t div_up(int64_t a, int64_t b) { return (a + b - 1) / b; }
int64_t align_up(int64_t a, int64_t b) { return div_up(a, b) * b; }

int check_geometry(const iga_patch_t* patch, int p, const iga_map_t* map, const iga_kappa_t* kappa, Geo& g)
{
    if (!patch || !map || !kappa) return fail(IGA_EINVAL, "patch, map and kappa must be non-null");
    if (patch->dim != 2 && patch->dim != 3) return fail(IGA_EUNSUPPORTED, "dim must be 2 or 3 (got %d)", patch->dim);
    if (p < 1 || p > kMaxP) return fail(IGA_EUNSUPPORTED, "degree p must be in 1..%d (got %d)", kMaxP, p);
    memset(&g, 0, sizeof(g));
    g.dim = patch->dim;
    g.p = p;
    for (int d = 0; d < 3; ++d) {
        if (d < g.dim) {
            if (patch->n_el[d] < p + 1)
                return fail(IGA_EINVAL, "n_el[%d] = %d: need at least p + 1 = %d elements (m >= 2p + 1)", d, patch->n_el[d], p + 1);
            if (patch->n_el[d] > (1 << 22)) return fail(IGA_EINVAL, "n_el[%d] too large", d);
            g.n_el[d] = patch->n_el[d];
            g.m[d] = patch->n_el[d] + p;
        } else {
            g.n_el[d] = 1;
            g.m[d] = 1;
        }
    }
    if (map->kind != IGA_MAP_IDENTITY && map->kind != IGA_MAP_AFFINE && map->kind != IGA_MAP_SINPROD)
        return fail(IGA_EINVAL, "unknown map kind %d", map->kind);
    g.map_kind = map->kind;
    g.amp = map->amp;
    for (int k = 0; k < 12; ++k) g.aff[k] = map->affine[k];
    switch (kappa->kind) {
    case IGA_KAPPA_CONST: case IGA_KAPPA_SIN2D: break;
    case IGA_KAPPA_EXPSIN3D:
        if (g.dim != 3) return fail(IGA_EINVAL, "IGA_KAPPA_EXPSIN3D needs dim 3");
        break;
    case IGA_KAPPA_POLY:
        if (kappa->deg < 0 || kappa->deg > 3) return fail(IGA_EINVAL, "polynomial kappa degree must be 0..3");
        break;
    case IGA_KAPPA_BSPLINE3:
        if (!kappa->ctrl) return fail(IGA_EINVAL, "IGA_KAPPA_BSPLINE3 needs a control value pointer");
        for (int d = 0; d < g.dim; ++d)
            if (kappa->nctrl[d] < 4 || kappa->nctrl[d] > 64)
                return fail(IGA_EINVAL, "IGA_KAPPA_BSPLINE3: nctrl[%d] = %d outside 4..64", d, kappa->nctrl[d]);
        break;
    default:
        return fail(IGA_EINVAL, "unknown kappa kind %d", kappa->kind);
    }
    g.kappa_kind = kappa->kind;
    g.kappa_deg = kappa->deg;
    g.ka = kappa->a;
    g.kb = kappa->b;
    for (int k = 0; k < 64; ++k) g.poly[k] = kappa->poly[k];
    if (kappa->kind == IGA_KAPPA_BSPLINE3) {
        for (int d = 0; d < 3; ++d) g.knc[d] = (d < g.dim) ? kappa->nctrl[d] : 1;
        g.kctrl = kappa->ctrl;
    }
    return IGA_OK;
}

void make_box(const Geo& g, Box& b, const int lo[3], const int R[3])
{
    memset(&b, 0, sizeof(b));
    for (int d = 0; d < 3; ++d) {
        if (d < g.dim) {
            b.rlo[d] = lo[d];
            b.R[d] = R[d];
            b.elo[d] = std::max(0, lo[d] - g.p);
            const int ehi = std::min(g.n_el[d] - 1, lo[d] + R[d] - 1);
            b.E[d] = ehi - b.elo[d] + 1;
        } else {
            b.rlo[d] = 0; b.R[d] = 1; b.elo[d] = 0; b.E[d] = 1;
        }
    }
}

struct Layout {
    int64_t total = 0;
    int64_t take(int64_t n_doubles) { int64_t o = total; total += align_up(std::max<int64_t>(n_doubles, 1), 32); return o; }
};

// Sample axis of one direction (SampleAxis in iga_internal.cuh).
SampleAxis common_axis(int k0, int k1, int M)
{
    SampleAxis a;
    memset(&a, 0, sizeof(a));
    a.c0 = k0; a.M = M; a.n_lo = 0; a.j_first = 0;
    a.n_mid = (k1 - k0) / M + 1;
    a.hi0 = k1;
    a.n_hi = ((k1 - k0) % M) ? 1 : 0;
    a.n = a.n_mid + a.n_hi;
    return a;
}

SampleAxis per_offset_axis(int p, int m, int M)
{
    SampleAxis a;
    memset(&a, 0, sizeof(a));
    const int c0 = p, c1 = m - p - 1;
    a.c0 = c0; a.M = M;
    if (c1 - c0 <= 2 * p + 1) {          // the two end runs meet: every cardinal index
        a.n_lo = c1 - c0 + 1;
        a.hi0 = c1 + 1;
    } else {
        a.n_lo = p + 1;
        a.j_first = p / M + 1;                      // first lattice point past the low run
        const int j_last = (c1 - p - 1 - c0) / M;   // last lattice point before the high run
        a.n_mid = std::max(0, j_last - a.j_first + 1);
        a.hi0 = c1 - p;
        a.n_hi = p + 1;
    }
    a.n = a.n_lo + a.n_mid + a.n_hi;
    return a;
}

// Interpolation plan (SplinePlan) of a surrogate: region of rows with
// interpolated entries [k0, k1] per direction -- the box Omega~ = [2p, m-2p-1]
// (Sec. 4), or the cardinal box [p, m-p-1] with per-offset domains (Sec. 3.2) --
// its sample axes and, per direction and offset component, the interpolation
// domain and samples.  empty = 1 when the region has no row.
int plan_spline(const Geo& g, int p, int M, int q, int domains, SplinePlan& sp, int& empty, int k1[3])
{
    const int dim = g.dim, W = 2 * p + 1;
    const int S = (dim == 3) ? W * W * W : W * W;
    memset(&sp, 0, sizeof(sp));
    sp.dim = dim; sp.q = q; sp.S = S; sp.c = (S - 1) / 2; sp.nv = W;
    // kernel-preserving surrogate (stiffness): upper offsets only, the diagonal is
    // minus the row sum; symmetric surrogate (mass): the diagonal is interpolated too
    sp.first = (g.form == kFormMass) ? sp.c : sp.c + 1;
    sp.all = (domains == IGA_DOMAINS_COMMON);
    empty = 0;
    const bool per_offset = (domains == IGA_DOMAINS_PER_OFFSET);
    const int k0 = per_offset ? p : 2 * p;
    for (int d = 0; d < dim; ++d) {
        k1[d] = g.m[d] - k0 - 1;
        if (k1[d] < k0) empty = 1;
    }
    if (empty) return IGA_OK;
    for (int d = 0; d < 3; ++d) {
        if (d >= dim) {
            sp.ax[d] = common_axis(0, 0, 1);
            sp.nu[d] = 1;
            sp.r0[d] = sp.r1[d] = 0;
            sp.Lmax[d] = 1;
            for (int v = 0; v < W; ++v) { sp.L[d][v] = 1; sp.ns[d][v] = 1; }
            continue;
        }
        sp.ax[d] = per_offset ? per_offset_axis(p, g.m[d], M) : common_axis(k0, k1[d], M);
        sp.nu[d] = sp.ax[d].n;
        if (sp.nu[d] > kMaxSamplesPerDir)
            return fail(IGA_EUNSUPPORTED, "more than %d samples per direction", kMaxSamplesPerDir);
        sp.r0[d] = k0;
        sp.r1[d] = k1[d];
        sp.Lmax[d] = 0;
        for (int v = 0; v < W; ++v) {
            const int dd = v - p;
            // domain of the offset component dd: Omega~_delta (Sec. 3.2) or Omega~
            const int lo = per_offset ? k0 + std::max(0, -dd) : k0;
            const int hi = per_offset ? k1[d] - std::max(0, dd) : k1[d];
            if (hi < lo) { sp.L[d][v] = 0; sp.ns[d][v] = 0; sp.k0[d][v] = lo; continue; }
            sp.k0[d][v] = lo;
            sp.L[d][v] = hi - lo + 1;
            int ns = 0;
            for (int a = 0; a < sp.nu[d]; ++a) ns += variant_sample(sp.ax[d], sp.all, axis_sample(sp.ax[d], a), lo, hi);
            sp.ns[d][v] = ns;
            sp.qe[d][v] = std::min(q, ns - 1);
            sp.Lmax[d] = std::max(sp.Lmax[d], sp.L[d][v]);
        }
    }
    sp.n_samples = 1;
    for (int d = 0; d < dim; ++d) sp.n_samples *= sp.nu[d];
    return IGA_OK;
}

// Scratch offsets of the interpolation tables of a plan.
struct SplineLayout {
    int64_t lu[3][kMaxV], eval[3][kMaxV], eval0[kMaxV], ints = 0;
    int64_t espan[3][kMaxV], pos[3][kMaxV], inv[3][kMaxV];
};

void spline_layout(Layout& lay, const SplinePlan& sp, SplineLayout& o)
{
    memset(&o, 0, sizeof(o));
    int64_t nints = 2 * 3 * kMaxV + 8;
    for (int d = 0; d < sp.dim; ++d)
        for (int v = 0; v < sp.nv; ++v) {
            const int64_t L = sp.L[d][v];
            o.lu[d][v] = lay.take((int64_t)sp.ns[d][v] * sp.ns[d][v]);
            o.eval[d][v] = lay.take(L * (sp.qe[d][v] + 1));
            if (d == 0) o.eval0[v] = lay.take(L * (sp.qe[d][v] + 1));
            o.espan[d][v] = nints;
            nints += align_up(L + 1, 8);
            o.pos[d][v] = nints;
            nints += align_up(sp.ns[d][v] + 1, 8);
            o.inv[d][v] = nints;
            nints += align_up(sp.nu[d] + 1, 8);
        }
    o.ints = lay.take(div_up(nints, 2));
}

void spline_bufs(double* scratch, const SplinePlan& sp, const SplineLayout& o, SplineBufs& sb)
{
    int* ints = (int*)(scratch + o.ints);
    sb.band = ints;
    for (int d = 0; d < sp.dim; ++d)
        for (int v = 0; v < sp.nv; ++v) {
            sb.lu[d][v] = scratch + o.lu[d][v];
            sb.eval[d][v] = scratch + o.eval[d][v];
            sb.espan[d][v] = ints + o.espan[d][v];
            sb.pos[d][v] = ints + o.pos[d][v];
            sb.inv[d][v] = ints + o.inv[d][v];
            if (d == 0) sb.eval0[v] = reinterpret_cast<float2*>(scratch + o.eval0[v]);
        }
}

}  // namespace

// One assembly split into its phases, so that a batch can run the quadrature
// stages of many patches as one persistent launch: plan (argument checks,
// boxes, sampling lattice, scratch layout, matrix storage), bind (scratch
// pointers), pre (tables, coefficient field), quad (sum-factorised stages),
// post (interpolation and fill).
struct iga::Job {
    Geo g;
    BoxSet bs;
    SplinePlan sp;
    SplineLayout slo;
    Layout lay;
    int empty = 0, dtype = 0, form = 0, arith = 0, tc64 = 0;
    bool do_spline = false, surrogate = false, created = false;
    int64_t nblk[4] = {0, 0, 0, 0};
    int64_t o_gx[3], o_sx[3], o_cx[3], o_wq[3], o_bv[3], o_bd[3], o_X[3], o_Xs[3], o_tdf[3];
    int64_t o_gshift = -1, o_ex_lo = -1, o_ex_hi = -1, o_samples = 0, o_partial = 0, o_mid = 0;
    int64_t o_kdf = -1, nctrl = 0;       // double-float copy of the B-spline coefficient's control values
    // mirror passes of the symmetric boxes: rows [begin, begin + count), +1 lower from upper, -1 upper from lower
    int n_mirror = 0;
    int64_t mir_begin[2] = {0, 0}, mir_count[2] = {0, 0};
    int mir_dir[2] = {0, 0};
    iga_matrix* A = nullptr;
    double* scratch = nullptr;
    double *gx[3], *sx[3], *cx[3], *wq[3], *bv[3], *bd[3], *X[3];
    void* Xs[3];
    float2* tdf[3];
    Tables T;
    SplineBufs sb;
    double* samples = nullptr;
};

namespace {

int job_plan(Job& J, const iga_patch_t* patch, int p, const iga_map_t* map, const iga_kappa_t* kappa, bool surrogate,
             int M, int q, int domains, int dtype, int form, iga_matrix* existing)
{
    Geo& g = J.g;
    int rc = check_geometry(patch, p, map, kappa, g);
    if (rc) return rc;
    g.form = form;
    J.form = form;
    J.dtype = dtype;
    J.surrogate = surrogate;
    if (form == kFormMass && domains != IGA_DOMAINS_COMMON)
        return fail(IGA_EUNSUPPORTED, "the mass surrogate uses the common domain Omega~");
    if (dtype != IGA_F64 && dtype != IGA_F32) return fail(IGA_EINVAL, "dtype must be IGA_F64 or IGA_F32");
    if (surrogate) {
        if (M < 1) return fail(IGA_EINVAL, "sampling parameter M must be >= 1 (got %d)", M);
        if (q < 0 || q > kMaxQ) return fail(IGA_EUNSUPPORTED, "interpolation degree q must be in 0..%d (got %d)", kMaxQ, q);
        if (domains != IGA_DOMAINS_COMMON && domains != IGA_DOMAINS_PER_OFFSET)
            return fail(IGA_EINVAL, "domains must be IGA_DOMAINS_COMMON or IGA_DOMAINS_PER_OFFSET (got %d)", domains);
    }
    const int dim = g.dim, W = 2 * p + 1, Q = p + 1, TT = Q * Q;
    const int S = (dim == 3) ? W * W * W : W * W;
    int64_t N = 1, nnz = 1;
    for (int d = 0; d < dim; ++d) {
        N *= g.m[d];
        nnz *= (int64_t)g.m[d] * W - (int64_t)p * (p + 1);
    }
    const size_t esz = (dtype == IGA_F32) ? 4 : 8;
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaGetDevice");

    iga_matrix* A = existing;
    if (A) {
        bool same = A->dim == dim && A->p == p && A->dtype == dtype && A->device == dev;
        for (int d = 0; d < dim; ++d) same = same && A->n_el[d] == g.n_el[d];
        if (!same) return fail(IGA_EINVAL, "matrix handle passed for reuse has another patch, degree, dtype or device");
    }

    // ---------------- plan: boxes and sampling lattice ----------------
    BoxSet& bs = J.bs;
    memset(&bs, 0, sizeof(bs));
    SplinePlan& sp = J.sp;
    memset(&sp, 0, sizeof(sp));
    std::vector<Box> boxes;
    if (surrogate) {
        const int k0 = (domains == IGA_DOMAINS_PER_OFFSET) ? p : 2 * p;
        int k1[3] = {0, 0, 0};
        rc = plan_spline(g, p, M, q, domains, sp, J.empty, k1);
        if (rc) return rc;
        if (!J.empty) {
            for (int d = 0; d < 3; ++d) bs.ax[d] = sp.ax[d];
            bs.n_samples = sp.n_samples;
            J.do_spline = true;
            // frame = rows with an index outside [k0, k1], as disjoint slabs
            Box b;
            if (dim == 3) {
                int lo[3], R[3];
                // slabs normal to direction 2
                lo[0] = 0; R[0] = g.m[0]; lo[1] = 0; R[1] = g.m[1];
                lo[2] = 0; R[2] = k0; make_box(g, b, lo, R); boxes.push_back(b);
                lo[2] = k1[2] + 1; R[2] = g.m[2] - 1 - k1[2]; make_box(g, b, lo, R); boxes.push_back(b);
                // normal to direction 1, inside the box in direction 2
                lo[2] = k0; R[2] = k1[2] - k0 + 1;
                lo[1] = 0; R[1] = k0; make_box(g, b, lo, R); boxes.push_back(b);
                lo[1] = k1[1] + 1; R[1] = g.m[1] - 1 - k1[1]; make_box(g, b, lo, R); boxes.push_back(b);
                // normal to direction 0
                lo[1] = k0; R[1] = k1[1] - k0 + 1;
                lo[0] = 0; R[0] = k0; make_box(g, b, lo, R); boxes.push_back(b);
                lo[0] = k1[0] + 1; R[0] = g.m[0] - 1 - k1[0]; make_box(g, b, lo, R); boxes.push_back(b);
            } else {
                int lo[3] = {0, 0, 0}, R[3] = {g.m[0], k0, 1};
                make_box(g, b, lo, R); boxes.push_back(b);
                lo[1] = k1[1] + 1; R[1] = g.m[1] - 1 - k1[1]; make_box(g, b, lo, R); boxes.push_back(b);
                lo[1] = k0; R[1] = k1[1] - k0 + 1;
                lo[0] = 0; R[0] = k0; make_box(g, b, lo, R); boxes.push_back(b);
                lo[0] = k1[0] + 1; R[0] = g.m[0] - 1 - k1[0]; make_box(g, b, lo, R); boxes.push_back(b);
            }
        }
    }
    if (!surrogate || J.empty) {
        Box b;
        int lo[3] = {0, 0, 0}, R[3] = {g.m[0], g.m[1], g.m[2]};
        make_box(g, b, lo, R);
        boxes.push_back(b);
    }
    if ((int)boxes.size() > kMaxBoxes) return fail(IGA_EINVAL, "internal: too many boxes");

    // ---------------- scratch layout ----------------
    Layout& lay = J.lay;
    const int arith = current_arith(dtype);
    J.arith = arith;
    for (int d = 0; d < 3; ++d) {
        const int64_t G = (d < dim) ? (int64_t)g.n_el[d] * Q : 1;
        const int64_t nX = (d < dim) ? (int64_t)4 * g.m[d] * W * TT : 1;
        J.o_gx[d] = lay.take(G); J.o_sx[d] = lay.take(2 * G); J.o_cx[d] = lay.take(2 * G); J.o_wq[d] = lay.take(G);
        J.o_bv[d] = lay.take(G * Q); J.o_bd[d] = lay.take(G * Q); J.o_X[d] = lay.take(nX);
        J.o_Xs[d] = (arith == kArithF64) ? J.o_X[d] : lay.take(nX);
        J.o_tdf[d] = lay.take(4 * G);
    }
    if (g.kappa_kind == IGA_KAPPA_BSPLINE3 && arith != kArithF64 && form == kFormStiffness) {
        J.nctrl = 1;
        for (int d = 0; d < dim; ++d) J.nctrl *= g.knc[d];
        J.o_kdf = lay.take(J.nctrl);                 // one float pair per control value
        g.kctrl_split = 1;
    }
    prepare_coef_df(g, arith);
    int64_t* nblk = J.nblk;
    bs.nb = (int)boxes.size();
    // FP64 values with tensor-core stage X: per-line T2 exponents of every box and the group shifts
    const int tc64 = (form == kFormStiffness && dtype == IGA_F64) ? current_tc(dtype) : 0;
    J.tc64 = tc64;
    if (tc64) J.o_gshift = lay.take(2);
    // The stiffness matrix is symmetric: boxes whose rows' partners i + delta on one side are rows of
    // the same box compute the other half of the offsets only, and a mirror pass copies the rest.
    // Exact (or a surrogate without Omega~): the whole patch (upper offsets).  Surrogate: the two
    // frame slabs normal to the slowest direction -- the low slab computes its upper offsets (every
    // lower partner lies in the slab), the high slab its lower ones.  Not with the tensor-core
    // stage X, which writes every offset of its rows.
    const bool sym_ok = form == kFormStiffness && !tc64 && !(dtype == IGA_F32 && current_tc(dtype));
    if (sym_ok && (!surrogate || J.empty)) {
        boxes[0].sym = 1;
        J.n_mirror = 1;
        J.mir_begin[0] = 0; J.mir_count[0] = N; J.mir_dir[0] = 1;
    } else if (sym_ok && surrogate && !J.empty && boxes.size() >= 2) {
        // boxes[0], boxes[1]: the slabs below and above Omega~ in the slowest direction, full in the others
        const int64_t plane = (dim == 3) ? (int64_t)g.m[0] * g.m[1] : (int64_t)g.m[0];
        boxes[0].sym = 1;
        boxes[1].sym = -1;
        J.n_mirror = 2;
        J.mir_begin[0] = (int64_t)boxes[0].rlo[dim - 1] * plane;
        J.mir_count[0] = (int64_t)boxes[0].R[dim - 1] * plane;
        J.mir_dir[0] = 1;
        J.mir_begin[1] = (int64_t)boxes[1].rlo[dim - 1] * plane;
        J.mir_count[1] = (int64_t)boxes[1].R[dim - 1] * plane;
        J.mir_dir[1] = -1;
    }
    for (int k = 0; k < bs.nb; ++k) {
        Box& b = boxes[k];
        b.out_kind = 0;
        b.ex_off = -1;
        if (tc64) {
            const int64_t lines = (dim == 3 ? (int64_t)b.R[2] * W : 1) * (int64_t)b.R[1] * W;
            b.ex_off = lay.take((lines + 1) / 2);
            if (J.o_ex_lo < 0) J.o_ex_lo = b.ex_off;
            J.o_ex_hi = lay.total;
        }
        b.c_off = lay.take(box_coef_len(dim, p, b));
        b.t1_off = lay.take(box_t1_len(dim, p, b));
        b.t2_off = lay.take(box_t2_len(dim, p, b));
        for (int st = 0; st < 4; ++st) {
            b.blk[st] = nblk[st];
            nblk[st] += div_up(box_items(dim, p, b, st), kBlock);
        }
        bs.box[k] = b;
    }
    if (J.do_spline) {
        Box sbx;                         // shape of every sample box: one row, p + 1 elements per direction
        memset(&sbx, 0, sizeof(sbx));
        for (int d = 0; d < 3; ++d) { sbx.R[d] = 1; sbx.E[d] = (d < dim) ? p + 1 : 1; }
        bs.s_c_len = align_up(box_coef_len(dim, p, sbx), 32);
        bs.s_t1_len = align_up(box_t1_len(dim, p, sbx), 32);
        bs.s_t2_len = align_up(box_t2_len(dim, p, sbx), 32);
        bs.s_c_off = lay.take(bs.s_c_len * sp.n_samples);
        bs.s_t1_off = lay.take(bs.s_t1_len * sp.n_samples);
        bs.s_t2_off = lay.take(bs.s_t2_len * sp.n_samples);
        for (int st = 0; st < 4; ++st) {
            bs.blk_s[st] = nblk[st];
            bs.bper_s[st] = div_up(box_items(dim, p, sbx, st), kBlock);
            nblk[st] += bs.bper_s[st] * sp.n_samples;
        }
        J.o_samples = lay.take((int64_t)S * sp.n_samples);
        spline_layout(lay, sp, J.slo);
        const int64_t S_up = S - sp.first;
        J.o_mid = lay.take(dim == 3 ? S_up * sp.Lmax[2] * (int64_t)sp.nu[1] * sp.nu[0] : 1);
        J.o_partial = lay.take(S_up * (dim == 3 ? sp.Lmax[2] : 1) * (int64_t)sp.Lmax[1] * sp.nu[0]);
    }
    for (int st = 0; st < 4; ++st)
        if (nblk[st] > 0x7fffffffLL) return fail(IGA_EUNSUPPORTED, "problem too large for one launch");

    // ---------------- storage ----------------
    if (!A) {
        A = new (std::nothrow) iga_matrix;
        if (!A) return fail(IGA_ENOMEM, "host allocation failed");
        memset(A, 0, sizeof(*A));
        A->dim = dim; A->p = p; A->dtype = dtype; A->device = dev;
        for (int d = 0; d < 3; ++d) { A->n_el[d] = g.n_el[d]; A->m[d] = g.m[d]; }
        A->N = N; A->S = S; A->nnz = nnz;
        A->bytes = (size_t)S * (size_t)N * esz;
        ce = cudaMalloc(&A->values, A->bytes);
        if (ce != cudaSuccess) { delete A; return cuda_fail(ce, "allocating matrix values"); }
        J.created = true;
    }
    J.A = A;
    return IGA_OK;
}

// Scratch pointers, tables and spline buffers of a planned job.
void job_bind(Job& J, double* scratch)
{
    J.scratch = scratch;
    auto P = [&](int64_t off) { return scratch + off; };
    for (int d = 0; d < 3; ++d) {
        J.gx[d] = P(J.o_gx[d]); J.sx[d] = P(J.o_sx[d]); J.cx[d] = P(J.o_cx[d]); J.wq[d] = P(J.o_wq[d]);
        J.bv[d] = P(J.o_bv[d]); J.bd[d] = P(J.o_bd[d]); J.X[d] = P(J.o_X[d]); J.Xs[d] = P(J.o_Xs[d]);
        J.tdf[d] = reinterpret_cast<float2*>(P(J.o_tdf[d]));
    }
    Tables& T = J.T;
    for (int d = 0; d < 3; ++d) {
        T.gx[d] = J.gx[d]; T.sx[d] = J.sx[d]; T.cx[d] = J.cx[d]; T.X[d] = J.X[d]; T.Xs[d] = J.Xs[d];
        T.tdf[d] = J.tdf[d];
    }
    T.arith = J.arith;
    T.tc = (J.dtype == IGA_F32) ? current_tc(J.dtype) : 0;
    T.tc64 = J.tc64;
    T.gshift = J.tc64 ? reinterpret_cast<const int*>(P(J.o_gshift)) : nullptr;
    J.samples = J.do_spline ? P(J.o_samples) : nullptr;
    J.g.kctrl_df = J.o_kdf >= 0 ? reinterpret_cast<const float2*>(P(J.o_kdf)) : nullptr;
    memset(&J.sb, 0, sizeof(J.sb));
    if (J.do_spline) {
        spline_bufs(scratch, J.sp, J.slo, J.sb);
        J.sb.partial = reinterpret_cast<float2*>(P(J.o_partial));
        J.sb.mid = P(J.o_mid);
    }
}

cudaError_t job_pre_impl(Job& J, cudaStream_t st, const char** stage)
{
    *stage = "basis tables";
    cudaError_t ce = launch_basis(J.g, J.gx, J.sx, J.cx, J.bv, J.bd, J.wq, J.tdf, st);
    if (ce == cudaSuccess && J.o_kdf >= 0) {
        *stage = "coefficient control values";
        ce = launch_split_ctrl(J.g.kctrl, J.nctrl, reinterpret_cast<float2*>(J.scratch + J.o_kdf), st);
    }
    if (ce == cudaSuccess) { *stage = "pair tables"; ce = launch_pairs(J.g, J.bv, J.bd, J.wq, J.X, J.Xs, J.arith, st); }
    if (ce == cudaSuccess && J.tc64) {
        *stage = "tensor-core stage X set-up";
        ce = launch_tc_group_shift(J.g, J.T, reinterpret_cast<int*>(J.scratch + J.o_gshift), st);
        if (ce == cudaSuccess && J.o_ex_lo >= 0)
            ce = cudaMemsetAsync(J.scratch + J.o_ex_lo, 0, (size_t)(J.o_ex_hi - J.o_ex_lo) * sizeof(double), st);
    }
    if (ce == cudaSuccess) { *stage = "coefficient field"; ce = launch_coef(J.g, J.T, J.bs, J.nblk[0], J.scratch, st); }
    return ce;
}

cudaError_t job_quad_impl(Job& J, cudaStream_t st, const char** stage)
{
    *stage = "quadrature stages";
    return (J.form == kFormMass)
               ? launch_mass_stages(J.g, J.T, J.bs, J.nblk, J.scratch, J.A->values, J.dtype == IGA_F32, J.samples, st)
               : launch_stages(J.g, J.T, J.bs, J.nblk, J.scratch, J.A->values, J.dtype == IGA_F32, J.samples, st);
}

cudaError_t job_post_impl(Job& J, cudaStream_t st, const char** stage)
{
    cudaError_t ce = cudaSuccess;
    for (int k = 0; k < J.n_mirror && ce == cudaSuccess; ++k) {
        *stage = "mirror of the symmetric matrix";
        ce = launch_mirror(J.g.dim, J.g.p, J.g.m, J.A->values, J.dtype == IGA_F32, J.mir_begin[k], J.mir_count[k],
                           J.mir_dir[k], st);
    }
    if (J.do_spline && ce == cudaSuccess) { *stage = "spline interpolation"; ce = launch_spline(J.g, J.sp, J.samples, J.sb, st); }
    if (J.surrogate && ce == cudaSuccess) {
        *stage = "surrogate fill";
        ce = launch_fill(J.g, J.sp, J.empty, J.sb, J.A->values, J.dtype == IGA_F32, st);
    }
    return ce;
}

void job_discard_matrix(Job& J)
{
    if (J.created && J.A) {
        cudaFree(J.A->values);
        delete J.A;
        J.A = nullptr;
        J.created = false;
    }
}

int assemble(const iga_patch_t* patch, int p, const iga_map_t* map, const iga_kappa_t* kappa, bool surrogate,
             int M, int q, int domains, int dtype, void* stream_v, iga_matrix_t* out, int form = kFormStiffness)
{
    t_err.clear();
    if (!out) return fail(IGA_EINVAL, "output handle pointer is null");
    Job J;
    int rc = job_plan(J, patch, p, map, kappa, surrogate, M, q, domains, dtype, form, *out);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream_v;
    cudaMemPool_t pool;
    cudaError_t ce = device_pool(J.A->device, &pool);
    if (ce != cudaSuccess) {
        job_discard_matrix(J);
        return cuda_fail(ce, "creating the memory pool");
    }
    double* scratch = nullptr;
    // inside a graph capture the allocation becomes a graph memory node (default pool)
    ce = t_capture ? cudaMallocAsync((void**)&scratch, (size_t)J.lay.total * sizeof(double), st)
                   : cudaMallocFromPoolAsync((void**)&scratch, (size_t)J.lay.total * sizeof(double), pool, st);
    if (ce != cudaSuccess) {
        job_discard_matrix(J);
        return cuda_fail(ce, "allocating scratch");
    }
    job_bind(J, scratch);
    const char* stage = "";
    ce = job_pre_impl(J, st, &stage);
    if (ce == cudaSuccess) ce = job_quad_impl(J, st, &stage);
    if (ce == cudaSuccess) ce = job_post_impl(J, st, &stage);
    cudaError_t fe = cudaFreeAsync(scratch, st);
    if (ce == cudaSuccess) ce = fe;
    if (ce != cudaSuccess) {
        job_discard_matrix(J);
        return cuda_fail(ce, stage);
    }
    *out = J.A;
    return IGA_OK;
}

}  // namespace

namespace iga {

void launch_begin(int kid, cudaStream_t s)
{
    (void)kid;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (g_profile.load(std::memory_order_relaxed) && !t_capture) {
        t_begin = take_event();
        if (t_begin) cudaEventRecord(t_begin, s);
    } else {
        t_begin = nullptr;
    }
}

int matrix_fields(iga_matrix_t A, int* dim, int* p, int m[3], int64_t* N, const void** vals, int* f32)
{
    if (!A) return fail(IGA_EINVAL, "null matrix");
    *dim = A->dim;
    *p = A->p;
    for (int d = 0; d < 3; ++d) m[d] = A->m[d];
    *N = A->N;
    *vals = A->values;
    *f32 = A->dtype == IGA_F32;
    return IGA_OK;
}

cudaError_t pool_alloc(size_t bytes, cudaStream_t s, void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaMemPool_t pool;
    if ((e = device_pool(dev, &pool)) != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(out, bytes, pool, s);
}

int current_arith(int dtype)
{
    return g_arith[dtype == IGA_F32 ? 1 : 0].load();
}

int current_tc(int dtype)
{
    if (dtype == IGA_F32) return g_arith[1].load() == kArithF32 ? g_tc_f32.load() : 0;
    return g_arith[0].load() == kArithDF ? g_tc_f64.load() : 0;
}

int report_error(int code, const char* msg)
{
    t_err = msg ? msg : "";
    return code;
}

void set_capture(bool on) { t_capture = on; }

int validate_geometry(const iga_patch_t* patch, int p, const iga_map_t* map, const iga_kappa_t* kappa, Geo& g)
{
    return check_geometry(patch, p, map, kappa, g);
}

void add_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int64_t launch_count() { return g_launches.load(); }

int assemble_patch(const iga_patch_t* patch, int p, const iga_map_t* map, const iga_kappa_t* kappa, bool surrogate,
                   int M, int q, int domains, int dtype, void* stream, iga_matrix_t* out)
{
    return assemble(patch, p, map, kappa, surrogate, M, q, domains, dtype, stream, out);
}

int job_create(const iga_patch_t* patch, int p, const iga_map_t* map, const iga_kappa_t* kappa, bool surrogate, int M,
               int q, int domains, int dtype, iga_matrix_t existing, Job** out)
{
    t_err.clear();
    Job* J = new (std::nothrow) Job;
    if (!J) return fail(IGA_ENOMEM, "host allocation failed");
    const int rc = job_plan(*J, patch, p, map, kappa, surrogate, M, q, domains, dtype, kFormStiffness, existing);
    if (rc) {
        delete J;
        return rc;
    }
    *out = J;
    return IGA_OK;
}

int64_t job_scratch_doubles(const Job* J) { return J->lay.total; }
void job_set_scratch(Job* J, double* scratch) { job_bind(*J, scratch); }
iga_matrix_t job_matrix(const Job* J) { return J->A; }

cudaError_t job_pre(Job* J, cudaStream_t s)
{
    const char* stage = "";
    return job_pre_impl(*J, s, &stage);
}
cudaError_t job_quad(Job* J, cudaStream_t s)
{
    const char* stage = "";
    return job_quad_impl(*J, s, &stage);
}
cudaError_t job_post(Job* J, cudaStream_t s)
{
    const char* stage = "";
    return job_post_impl(*J, s, &stage);
}

bool job_persist_work(const Job* J, PersistWork* w)
{
    if (J->form != kFormStiffness || J->T.tc || J->T.tc64) return false;
    memset(w, 0, sizeof(*w));
    w->g = J->g;
    w->T = J->T;
    w->bs = J->bs;
    w->scratch = J->scratch;
    w->ell = J->A->values;
    w->ell_f32 = J->dtype == IGA_F32;
    w->N = J->A->N;
    w->samples = J->samples;
    for (int k = 0; k < 4; ++k) w->nb[k] = J->nblk[k];
    return true;
}

int job_dim(const Job* J) { return J->g.dim; }
int job_degree(const Job* J) { return J->g.p; }
int job_arith(const Job* J) { return J->arith; }

void job_destroy(Job* J, bool discard_new_matrix)
{
    if (!J) return;
    if (discard_new_matrix) job_discard_matrix(*J);
    delete J;
}

void launch_end(int kid, cudaStream_t s)
{
    if (!t_begin) return;
    cudaEvent_t e = take_event();
    if (!e) return;
    cudaEventRecord(e, s);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_pending.push_back({kid, t_begin, e});
    t_begin = nullptr;
}

}  // namespace iga

extern "C" {

int iga_assemble_exact(const iga_patch_t* patch, int p, const iga_map_t* map, const iga_kappa_t* kappa,
                       int dtype, void* stream, iga_matrix_t* A)
{
    return assemble(patch, p, map, kappa, false, 1, 0, IGA_DOMAINS_COMMON, dtype, stream, A);
}

int iga_assemble_surrogate(const iga_patch_t* patch, int p, const iga_map_t* map, const iga_kappa_t* kappa,
                           int M, int q, int dtype, void* stream, iga_matrix_t* A)
{
    return assemble(patch, p, map, kappa, true, M, q, IGA_DOMAINS_COMMON, dtype, stream, A);
}

int iga_assemble_mass(const iga_patch_t* patch, int p, const iga_map_t* map, int dtype, void* stream, iga_matrix_t* A)
{
    iga_kappa_t unit;
    memset(&unit, 0, sizeof(unit));
    unit.kind = IGA_KAPPA_CONST;
    unit.a = 1.0;
    return assemble(patch, p, map, &unit, false, 1, 0, IGA_DOMAINS_COMMON, dtype, stream, A, kFormMass);
}

int iga_assemble_mass_surrogate(const iga_patch_t* patch, int p, const iga_map_t* map, int M, int q, int dtype,
                                void* stream, iga_matrix_t* A)
{
    iga_kappa_t unit;
    memset(&unit, 0, sizeof(unit));
    unit.kind = IGA_KAPPA_CONST;
    unit.a = 1.0;
    return assemble(patch, p, map, &unit, true, M, q, IGA_DOMAINS_COMMON, dtype, stream, A, kFormMass);
}

int iga_surrogate_plan(const iga_patch_t* patch, int p, int M, int q, int domains, int cap, int32_t* samples,
                       int32_t* n_samples, int32_t* dom_lo, int32_t* dom_hi, int32_t* dom_ns, int32_t* dom_q,
                       int* empty)
{
    t_err.clear();
    iga_map_t map;
    memset(&map, 0, sizeof(map));
    map.kind = IGA_MAP_IDENTITY;
    iga_kappa_t unit;
    memset(&unit, 0, sizeof(unit));
    unit.kind = IGA_KAPPA_CONST;
    unit.a = 1.0;
    Geo g;
    int rc = check_geometry(patch, p, &map, &unit, g);       // the patch and degree checks of the assembly
    if (rc) return rc;
    if (M < 1) return fail(IGA_EINVAL, "sampling parameter M must be >= 1 (got %d)", M);
    if (q < 0 || q > kMaxQ) return fail(IGA_EUNSUPPORTED, "interpolation degree q must be in 0..%d (got %d)", kMaxQ, q);
    if (domains != IGA_DOMAINS_COMMON && domains != IGA_DOMAINS_PER_OFFSET)
        return fail(IGA_EINVAL, "domains must be IGA_DOMAINS_COMMON or IGA_DOMAINS_PER_OFFSET (got %d)", domains);
    if (!samples || !n_samples || !empty || cap < 1) return fail(IGA_EINVAL, "samples, n_samples and empty must be non-null, cap >= 1");
    const bool doms = dom_lo || dom_hi || dom_ns || dom_q;
    if (doms && !(dom_lo && dom_hi && dom_ns && dom_q)) return fail(IGA_EINVAL, "dom_lo, dom_hi, dom_ns, dom_q: all or none");
    g.form = kFormStiffness;
    SplinePlan sp;
    int emp = 0, k1[3] = {0, 0, 0};
    rc = plan_spline(g, p, M, q, domains, sp, emp, k1);
    if (rc) return rc;
    *empty = emp;
    if (emp) return IGA_OK;
    for (int d = 0; d < 3; ++d)
        if (sp.nu[d] > cap) return fail(IGA_EINVAL, "direction %d has %d samples, more than cap = %d", d, sp.nu[d], cap);
    for (int d = 0; d < 3; ++d) {
        n_samples[d] = sp.nu[d];
        for (int a = 0; a < sp.nu[d]; ++a) samples[(int64_t)d * cap + a] = axis_sample(sp.ax[d], a);
    }
    if (doms) {
        const int W = 2 * p + 1;
        for (int d = 0; d < 3; ++d)
            for (int v = 0; v < W; ++v) {
                const int k = d * W + v;
                const bool real = d < g.dim;
                dom_lo[k] = real ? sp.k0[d][v] : 0;
                dom_hi[k] = real ? sp.k0[d][v] + sp.L[d][v] - 1 : 0;
                dom_ns[k] = real ? sp.ns[d][v] : 1;
                dom_q[k] = (real && sp.ns[d][v] > 0) ? sp.qe[d][v] : 0;
            }
    }
    return IGA_OK;
}

int iga_kappa_gradient(const iga_patch_t* patch, int p, const iga_map_t* map, const iga_kappa_t* kappa, int M,
                       int q, const double* ybar, const double* x, double* grad, void* stream_v)
{
    t_err.clear();
    Geo g;
    int rc = check_geometry(patch, p, map, kappa, g);
    if (rc) return rc;
    if (kappa->kind != IGA_KAPPA_BSPLINE3) return fail(IGA_EINVAL, "the kappa gradient needs IGA_KAPPA_BSPLINE3");
    if (!ybar || !x || !grad) return fail(IGA_EINVAL, "ybar, x and grad must be non-null device pointers");
    if (M < 0) return fail(IGA_EINVAL, "M must be 0 (exact matrix) or >= 1 (surrogate), got %d", M);
    if (M >= 1 && (q < 0 || q > kMaxQ))
        return fail(IGA_EUNSUPPORTED, "interpolation degree q must be in 0..%d (got %d)", kMaxQ, q);
    const int dim = g.dim, Q = p + 1;
    int64_t N = 1, nctrl = 1, npts = 1;
    int64_t G[3] = {1, 1, 1};
    for (int d = 0; d < dim; ++d) {
        N *= g.m[d];
        nctrl *= g.knc[d];
        G[d] = (int64_t)g.n_el[d] * Q;
        npts *= G[d];
    }
    cudaStream_t st = (cudaStream_t)stream_v;
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaGetDevice");

    SplinePlan sp;
    memset(&sp, 0, sizeof(sp));
    int empty = 1, k1[3] = {0, 0, 0};
    if (M >= 1) {
        rc = plan_spline(g, p, M, q, IGA_DOMAINS_COMMON, sp, empty, k1);
        if (rc) return rc;
    }
    const bool sur = (M >= 1) && !empty;       // an empty Omega~ leaves the exact matrix

    // ---------------- scratch ----------------
    Layout lay;
    int64_t o_gx[3], o_sx[3], o_cx[3], o_wq[3], o_bv[3], o_bd[3], o_tdf[3];
    for (int d = 0; d < 3; ++d) {
        const int64_t Gd = (d < dim) ? G[d] : 1;
        o_gx[d] = lay.take(Gd); o_sx[d] = lay.take(2 * Gd); o_cx[d] = lay.take(2 * Gd); o_wq[d] = lay.take(Gd);
        o_bv[d] = lay.take(Gd * Q); o_bd[d] = lay.take(Gd * Q); o_tdf[d] = lay.take(4 * Gd);
    }
    const int64_t m2 = (dim == 3) ? g.m[2] : 1;
    const int64_t tot0 = m2 * g.m[1] * G[0], tot1 = m2 * G[1] * G[0];
    const int nvec = sur ? 6 : 2;
    const int64_t o_W0 = lay.take(2 * tot0);
    int64_t o_W1[6];
    for (int v = 0; v < nvec; ++v) o_W1[v] = lay.take(3 * tot1);
    const int64_t o_vec = sur ? lay.take(4 * N) : 0;
    const int64_t o_spt = lay.take(npts);
    SplineLayout slo;
    int64_t o_C0 = 0, o_C1 = 0, o_tab = 0;
    if (sur) {
        spline_layout(lay, sp, slo);
        const int P = p;
        const int64_t S_up = sp.S - sp.first;
        const int64_t L1 = sp.L[1][P], L2 = (dim == 3) ? sp.L[2][P] : 1;
        o_C0 = lay.take(S_up * L2 * L1 * sp.nu[0]);
        o_C1 = lay.take(dim == 3 ? S_up * L2 * (int64_t)sp.nu[1] * sp.nu[0] : 1);
        o_tab = lay.take(S_up * sp.n_samples);
    }
    cudaMemPool_t pool;
    if ((ce = device_pool(dev, &pool)) != cudaSuccess) return cuda_fail(ce, "creating the memory pool");
    double* scratch = nullptr;
    ce = cudaMallocFromPoolAsync((void**)&scratch, (size_t)lay.total * sizeof(double), pool, st);
    if (ce != cudaSuccess) return cuda_fail(ce, "allocating scratch");
    auto P = [&](int64_t off) { return scratch + off; };

    // ---------------- launches ----------------
    double *gx[3], *sx[3], *cx[3], *wq[3], *bv[3], *bd[3];
    float2* tdf[3];
    AdjTables T;
    for (int d = 0; d < 3; ++d) {
        gx[d] = P(o_gx[d]); sx[d] = P(o_sx[d]); cx[d] = P(o_cx[d]); wq[d] = P(o_wq[d]);
        bv[d] = P(o_bv[d]); bd[d] = P(o_bd[d]); tdf[d] = reinterpret_cast<float2*>(P(o_tdf[d]));
        T.gx[d] = gx[d]; T.sx[d] = sx[d]; T.cx[d] = cx[d]; T.wq[d] = wq[d]; T.bv[d] = bv[d]; T.bd[d] = bd[d];
    }
    const char* stage = "basis tables";
    ce = launch_basis(g, gx, sx, cx, bv, bd, wq, tdf, st);
    // vectors whose bilinear forms carry the exact entries
    const double* vecs[6] = {ybar, x, nullptr, nullptr, nullptr, nullptr};
    if (sur && ce == cudaSuccess) {
        stage = "restricted vectors";
        ce = launch_adj_vectors(g, sp, ybar, x, P(o_vec), st);
        for (int k = 0; k < 4; ++k) vecs[2 + k] = P(o_vec) + k * N;
    }
    for (int v = 0; v < nvec && ce == cudaSuccess; ++v) {
        stage = "gradient fields";
        ce = launch_adj_grad_field(g, T, vecs[v], P(o_W0), P(o_W1[v]), st);
    }
    AdjTerms terms;
    memset(&terms, 0, sizeof(terms));
    terms.tot1 = tot1;
    terms.n = sur ? 3 : 1;
    terms.sign[0] = 1.0; terms.Wa[0] = P(o_W1[0]); terms.Wb[0] = P(o_W1[1]);
    if (sur) {
        terms.sign[1] = -1.0; terms.Wa[1] = P(o_W1[2]); terms.Wb[1] = P(o_W1[3]);
        terms.sign[2] = 1.0; terms.Wa[2] = P(o_W1[4]); terms.Wb[2] = P(o_W1[5]);
    }
    if (ce == cudaSuccess) { stage = "point field"; ce = launch_adj_points(g, T, terms, P(o_spt), st); }
    if (sur) {
        SplineBufs sb;
        memset(&sb, 0, sizeof(sb));
        spline_bufs(scratch, sp, slo, sb);
        if (ce == cudaSuccess) { stage = "spline tables"; ce = launch_spline_setup(sp, sb, st); }
        if (ce == cudaSuccess) {
            stage = "transposed interpolation";
            ce = launch_adj_interp(g, sp, sb, ybar, x, P(o_C0), P(o_C1), P(o_tab), st);
        }
        if (ce == cudaSuccess) { stage = "sample rows"; ce = launch_adj_samples(g, T, sp, P(o_tab), P(o_spt), st); }
    }
    if (ce == cudaSuccess) { stage = "gradient reset"; ce = cudaMemsetAsync(grad, 0, (size_t)nctrl * sizeof(double), st); }
    if (ce == cudaSuccess) { stage = "control scatter"; ce = launch_adj_scatter(g, T, P(o_spt), grad, st); }
    cudaError_t fe = cudaFreeAsync(scratch, st);
    if (ce == cudaSuccess) ce = fe;
    if (ce != cudaSuccess) return cuda_fail(ce, stage);
    return IGA_OK;
}

int iga_manufactured_load(const iga_patch_t* patch, int p, const iga_map_t* map, const iga_kappa_t* kappa, int freq,
                          double* F, double* energy, void* stream_v)
{
    t_err.clear();
    Geo g;
    int rc = check_geometry(patch, p, map, kappa, g);
    if (rc) return rc;
    if (!F || !energy) return fail(IGA_EINVAL, "F and energy must be non-null device pointers");
    if (freq < 1 || freq > 1000) return fail(IGA_EINVAL, "frequency k must be in 1..1000 (got %d)", freq);
    const int dim = g.dim, Q = p + 1;
    int64_t npts = 1;
    for (int d = 0; d < dim; ++d) npts *= (int64_t)g.n_el[d] * Q;
    const int64_t npart = npts / (8 * kBlock) + 2;
    cudaStream_t st = (cudaStream_t)stream_v;
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaGetDevice");
    Layout lay;
    int64_t o_gx[3], o_sx[3], o_cx[3], o_wq[3], o_bv[3], o_bd[3], o_tdf[3];
    for (int d = 0; d < 3; ++d) {
        const int64_t G = (d < dim) ? (int64_t)g.n_el[d] * Q : 1;
        o_gx[d] = lay.take(G); o_sx[d] = lay.take(2 * G); o_cx[d] = lay.take(2 * G); o_wq[d] = lay.take(G);
        o_bv[d] = lay.take(G * Q); o_bd[d] = lay.take(G * Q); o_tdf[d] = lay.take(4 * G);
    }
    const int64_t o_V = lay.take(dim * npts), o_E = lay.take(npts), o_part = lay.take(2 * npart);
    cudaMemPool_t pool;
    if ((ce = device_pool(dev, &pool)) != cudaSuccess) return cuda_fail(ce, "creating the memory pool");
    double* scratch = nullptr;
    ce = cudaMallocFromPoolAsync((void**)&scratch, (size_t)lay.total * sizeof(double), pool, st);
    if (ce != cudaSuccess) return cuda_fail(ce, "allocating scratch");
    double *gx[3], *sx[3], *cx[3], *wq[3], *bv[3], *bd[3];
    float2* tdf[3];
    MmsArgs A;
    for (int d = 0; d < 3; ++d) {
        gx[d] = scratch + o_gx[d]; sx[d] = scratch + o_sx[d]; cx[d] = scratch + o_cx[d]; wq[d] = scratch + o_wq[d];
        bv[d] = scratch + o_bv[d]; bd[d] = scratch + o_bd[d]; tdf[d] = reinterpret_cast<float2*>(scratch + o_tdf[d]);
        A.gx[d] = gx[d]; A.wq[d] = wq[d]; A.bv[d] = bv[d]; A.bd[d] = bd[d];
    }
    A.V = scratch + o_V;
    A.E = scratch + o_E;
    A.freq = freq;
    const char* stage = "basis tables";
    ce = launch_basis(g, gx, sx, cx, bv, bd, wq, tdf, st);
    if (ce == cudaSuccess) { stage = "manufactured load"; ce = launch_manufactured(g, A, F, energy, scratch + o_part, npart, st); }
    cudaError_t fe = cudaFreeAsync(scratch, st);
    if (ce == cudaSuccess) ce = fe;
    if (ce != cudaSuccess) return cuda_fail(ce, stage);
    return IGA_OK;
}

int iga_assemble_surrogate_domains(const iga_patch_t* patch, int p, const iga_map_t* map, const iga_kappa_t* kappa,
                                   int M, int q, int domains, int dtype, void* stream, iga_matrix_t* A)
{
    return assemble(patch, p, map, kappa, true, M, q, domains, dtype, stream, A);
}

int iga_apply(iga_matrix_t A, const void* x, void* y, void* stream)
{
    t_err.clear();
    if (!A || !x || !y) return fail(IGA_EINVAL, "iga_apply: null argument");
    if (x == y) return fail(IGA_EINVAL, "iga_apply: x and y must not overlap");
    cudaError_t e = launch_spmv(A->dim, A->p, A->m, A->values, A->dtype == IGA_F32, x, y, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "stencil SpMV");
    return IGA_OK;
}

int iga_apply_host(iga_matrix_t A, const void* x_host, void* y_host, void* stream)
{
    t_err.clear();
    if (!A || !x_host || !y_host) return fail(IGA_EINVAL, "iga_apply_host: null argument");
    cudaStream_t st = (cudaStream_t)stream;
    cudaMemPool_t pool;
    cudaError_t e = device_pool(A->device, &pool);
    if (e != cudaSuccess) return cuda_fail(e, "memory pool");
    const size_t vb = (size_t)A->N * (A->dtype == IGA_F32 ? 4 : 8);
    void* buf = nullptr;
    e = cudaMallocFromPoolAsync(&buf, 2 * align_up((int64_t)vb, 256), pool, st);
    if (e != cudaSuccess) return cuda_fail(e, "staging buffers");
    void* dx = buf;
    void* dy = (char*)buf + align_up((int64_t)vb, 256);
    e = cudaMemcpyAsync(dx, x_host, vb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_spmv(A->dim, A->p, A->m, A->values, A->dtype == IGA_F32, dx, dy, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(y_host, dy, vb, cudaMemcpyDeviceToHost, st);
    cudaError_t fe = cudaFreeAsync(buf, st);
    cudaError_t se = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = fe;
    if (e == cudaSuccess) e = se;
    if (e != cudaSuccess) return cuda_fail(e, "iga_apply_host");
    return IGA_OK;
}

int iga_matrix_info(iga_matrix_t A, int64_t* N, int32_t* S, int64_t* nnz, int32_t* dtype)
{
    t_err.clear();
    if (!A) return fail(IGA_EINVAL, "null matrix");
    if (N) *N = A->N;
    if (S) *S = A->S;
    if (nnz) *nnz = A->nnz;
    if (dtype) *dtype = A->dtype;
    return IGA_OK;
}

int iga_matrix_values(iga_matrix_t A, const void** values)
{
    t_err.clear();
    if (!A || !values) return fail(IGA_EINVAL, "null argument");
    *values = A->values;
    return IGA_OK;
}

int iga_matrix_copy_values(iga_matrix_t A, void* dst, int dst_on_host, void* stream)
{
    t_err.clear();
    if (!A || !dst) return fail(IGA_EINVAL, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(dst, A->values, A->bytes,
                                    dst_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "copying values");
    return IGA_OK;
}

int iga_matrix_destroy(iga_matrix_t A)
{
    t_err.clear();
    if (!A) return IGA_OK;
    batch_forget(A);                 // cached batch graphs write into this matrix: drop them
    cudaError_t e = cudaFree(A->values);
    delete A;
    if (e != cudaSuccess) return cuda_fail(e, "freeing matrix values");
    return IGA_OK;
}

int iga_set_arithmetic(int dtype, int arith)
{
    t_err.clear();
    if (dtype != IGA_F64 && dtype != IGA_F32) return fail(IGA_EINVAL, "dtype must be IGA_F64 or IGA_F32");
    int a, tc = 0;
    switch (arith) {
    case IGA_ARITH_FP64: a = kArithF64; break;
    case IGA_ARITH_DF64: a = kArithDF; break;
    case IGA_ARITH_FP32: a = kArithF32; break;
    case IGA_ARITH_BF16X3: a = kArithF32; tc = 1; break;
    case IGA_ARITH_DF64_TC: a = kArithDF; tc = 1; break;
    default: return fail(IGA_EINVAL, "unknown arithmetic %d", arith);
    }
    if (arith == IGA_ARITH_BF16X3 && dtype != IGA_F32)
        return fail(IGA_EINVAL, "IGA_ARITH_BF16X3 is for IGA_F32 values (use IGA_ARITH_DF64_TC for IGA_F64)");
    if (arith == IGA_ARITH_DF64_TC && dtype != IGA_F64)
        return fail(IGA_EINVAL, "IGA_ARITH_DF64_TC is for IGA_F64 values (use IGA_ARITH_BF16X3 for IGA_F32)");
    if (dtype == IGA_F64 && a == kArithF32)
        return fail(IGA_EINVAL, "FP32 contractions cannot meet FP64 accuracy; use IGA_ARITH_FP64 or IGA_ARITH_DF64");
    g_arith[dtype == IGA_F32 ? 1 : 0].store(a);
    if (dtype == IGA_F32) g_tc_f32.store(tc);
    else g_tc_f64.store(tc);
    return IGA_OK;
}

int iga_get_arithmetic(int dtype)
{
    const int a = current_arith(dtype);
    if (current_tc(dtype)) return dtype == IGA_F32 ? IGA_ARITH_BF16X3 : IGA_ARITH_DF64_TC;
    return a == kArithF64 ? IGA_ARITH_FP64 : a == kArithDF ? IGA_ARITH_DF64 : IGA_ARITH_FP32;
}

int64_t iga_launch_count(void) { return g_launches.load(); }

int iga_profile_enable(int on)
{
    g_profile.store(on ? 1 : 0);
    return IGA_OK;
}

int iga_profile_read(int n, int64_t* launches, double* ms)
{
    t_err.clear();
    if (n < 0 || (n > 0 && (!launches || !ms))) return fail(IGA_EINVAL, "iga_profile_read: bad arguments");
    for (int k = 0; k < n; ++k) { launches[k] = 0; ms[k] = 0.0; }
    std::vector<Pending> pend;
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        pend.swap(g_pending);
    }
    int rc = IGA_OK;
    for (auto& pd : pend) {
        float t = 0.f;
        cudaError_t e = cudaEventSynchronize(pd.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, pd.a, pd.b);
        if (e != cudaSuccess) rc = cuda_fail(e, "reading profile events");
        else if (pd.kid < n) { launches[pd.kid] += 1; ms[pd.kid] += t; }
    }
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto& pd : pend) { g_events.push_back(pd.a); g_events.push_back(pd.b); }
    return rc;
}

int iga_num_kernels(void) { return K_NUM; }

const char* iga_kernel_name(int k) { return (k >= 0 && k < K_NUM) ? kNames[k] : ""; }

const char* iga_last_error(void) { return t_err.c_str(); }

int iga_version(void) { return 10000; }

}  // extern "C"
