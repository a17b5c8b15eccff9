// iga_assemble_exact_noalloc: exact assembly for callers that cannot allocate
// device memory.
//
// Some callers must not allocate during a call: code running inside a
// real-time or latency-critical loop where cudaMalloc/cudaFree would
// synchronise the device or stall, applications that hand the GPU's memory to
// their own allocator and forbid other allocations, and environments that
// cap or forbid allocation after start-up.  This entry point gives them the
// exact assembly with no allocation at all: the caller passes the output
// values buffer, and the scratch the quadrature needs (basis and pair tables,
// coefficient field, the two contraction intermediates) lives in one
// file-scope device array of fixed size, reserved on every GPU that loads
// this library until the process exits.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "arith.cuh"
#include "iga_internal.cuh"

namespace {

// Maximum scratch of the no-allocation path: 64 MiB (8 Mi doubles).
constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchBytes / sizeof(double)];

// Failures are reported through iga_last_error() like every other call.
int noalloc_fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    return iga::report_error(code, buf);
}

// Device address of g_noalloc_scratch per device, looked up once per device
// (with that device current) by the first call on it.  The cached address
// belongs to the device's primary context: it is not valid after
// cudaDeviceReset() or any other teardown of that context, and calls made
// after one would launch against a stale address.
std::mutex g_sym_mu;
double* g_sym_addr[128] = {};

int scratch_address(int dev, double** out)
{
    if (dev < 0 || dev >= 128) return noalloc_fail(IGA_EINVAL, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_sym_mu);
    if (!g_sym_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return noalloc_fail(IGA_ECUDA, "cudaGetSymbolAddress of the no-allocation scratch failed: %s",
                                cudaGetErrorString(e));
        g_sym_addr[dev] = (double*)p;
    }
    *out = g_sym_addr[dev];
    return IGA_OK;
}

int64_t up32(int64_t n) { return ((n > 0 ? n : 1) + 31) / 32 * 32; }

}  // namespace

using namespace iga;

extern "C" int iga_assemble_exact_noalloc(const iga_patch_t* patch, int p, const iga_map_t* map,
                                          const iga_kappa_t* kappa, int dtype, void* values, void* stream)
{
    iga::report_error(IGA_OK, "");
    // the argument checks of iga_assemble_exact (every map and coefficient kind,
    // B-spline coefficients included: their control values are the caller's)
    Geo g;
    int rc = validate_geometry(patch, p, map, kappa, g);
    if (rc) return rc;
    if (!values) return noalloc_fail(IGA_EINVAL, "values must be a non-null device pointer");
    if (dtype != IGA_F64 && dtype != IGA_F32) return noalloc_fail(IGA_EINVAL, "dtype must be IGA_F64 or IGA_F32");

    // one box: every row of the patch
    const int Q = p + 1, W = 2 * p + 1, TT = Q * Q;
    BoxSet bs;
    memset(&bs, 0, sizeof(bs));
    bs.nb = 1;
    Box& b = bs.box[0];
    for (int d = 0; d < 3; ++d) {
        b.rlo[d] = 0;
        b.R[d] = g.m[d];
        b.elo[d] = 0;
        b.E[d] = g.n_el[d];
    }
    // scratch layout (doubles, 256-byte aligned pieces)
    int64_t off = 0;
    const int arith = current_arith(dtype);
    int64_t o_gx[3], o_sx[3], o_cx[3], o_wq[3], o_bv[3], o_bd[3], o_X[3], o_Xs[3], o_tdf[3];
    for (int d = 0; d < 3; ++d) {
        const int64_t G = (d < g.dim) ? (int64_t)g.n_el[d] * Q : 1;
        const int64_t nX = (d < g.dim) ? (int64_t)4 * g.m[d] * W * TT : 1;
        o_gx[d] = off; off += up32(G);
        o_sx[d] = off; off += up32(2 * G);
        o_cx[d] = off; off += up32(2 * G);
        o_wq[d] = off; off += up32(G);
        o_bv[d] = off; off += up32(G * Q);
        o_bd[d] = off; off += up32(G * Q);
        o_X[d] = off; off += up32(nX);
        if (arith == kArithF64) o_Xs[d] = o_X[d];
        else { o_Xs[d] = off; off += up32(nX); }
        o_tdf[d] = off; off += up32(4 * G);
    }
    prepare_coef_df(g, arith);
    b.out_kind = 0;
    b.ex_off = -1;
    b.c_off = off; off += up32(box_coef_len(g.dim, p, b));
    b.t1_off = off; off += up32(box_t1_len(g.dim, p, b));
    b.t2_off = off; off += up32(box_t2_len(g.dim, p, b));
    const int64_t need = off * (int64_t)sizeof(double);
    if (need > (int64_t)kNoAllocScratchBytes)
        return noalloc_fail(IGA_EUNSUPPORTED,
                            "this patch needs %lld bytes of quadrature scratch; the no-allocation entry point "
                            "holds at most %llu bytes (64 MiB): use iga_assemble_exact",
                            (long long)need, (unsigned long long)kNoAllocScratchBytes);
    int64_t nblk[4] = {0, 0, 0, 0};
    for (int s = 0; s < 4; ++s) {
        b.blk[s] = 0;
        nblk[s] = (box_items(g.dim, p, b, s) + kBlock - 1) / kBlock;
        if (nblk[s] > 0x7fffffffLL) return noalloc_fail(IGA_EUNSUPPORTED, "problem too large for one launch");
    }

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(IGA_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    double* scratch = nullptr;
    rc = scratch_address(dev, &scratch);
    if (rc) return rc;

    cudaStream_t st = (cudaStream_t)stream;
    double *gx[3], *sx[3], *cx[3], *wq[3], *bv[3], *bd[3], *X[3];
    void* Xs[3];
    float2* tdf[3];
    for (int d = 0; d < 3; ++d) {
        gx[d] = scratch + o_gx[d]; sx[d] = scratch + o_sx[d]; cx[d] = scratch + o_cx[d];
        wq[d] = scratch + o_wq[d]; bv[d] = scratch + o_bv[d]; bd[d] = scratch + o_bd[d]; X[d] = scratch + o_X[d];
        Xs[d] = scratch + o_Xs[d];
        tdf[d] = reinterpret_cast<float2*>(scratch + o_tdf[d]);
    }
    Tables T;
    for (int d = 0; d < 3; ++d) {
        T.gx[d] = gx[d]; T.sx[d] = sx[d]; T.cx[d] = cx[d]; T.X[d] = X[d]; T.Xs[d] = Xs[d]; T.tdf[d] = tdf[d];
    }
    T.arith = arith;
    T.tc = (dtype == IGA_F32) ? current_tc(dtype) : 0;
    T.tc64 = 0;                       // the FP64 tensor-core stage needs per-line exponent scratch
    T.gshift = nullptr;
    e = launch_basis(g, gx, sx, cx, bv, bd, wq, tdf, st);
    if (e == cudaSuccess) e = launch_pairs(g, bv, bd, wq, X, Xs, arith, st);
    if (e == cudaSuccess) e = launch_coef(g, T, bs, nblk[0], scratch, st);
    if (e == cudaSuccess) e = launch_stages(g, T, bs, nblk, scratch, values, dtype == IGA_F32, nullptr, st);
    if (e != cudaSuccess) return noalloc_fail(IGA_ECUDA, "no-allocation exact assembly: %s", cudaGetErrorString(e));
    return IGA_OK;
}
