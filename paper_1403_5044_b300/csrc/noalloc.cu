// swj_residual_noalloc: the residual E(u) for callers that cannot allocate
// device memory.
//
// Some hosts hand this library only the buffers they already own and must not
// see the library allocate: a serving loop with a fixed latency budget
// (cudaMalloc and cudaFree synchronise the whole device and stall every other
// stream) or an embedding framework that budgets all device memory up front
// and forbids allocation after start-up.  For them this entry point computes
// what swj_residual computes with default options (source forcing), with the
// same kernels, but takes its scratch (mesh-step arrays, pair records,
// per-chunk partial sums) from one file-scope device array instead of a
// context's cudaMalloc'ed workspace.  When the partial sums of the context's
// launch plan do not fit, it uses fewer source chunks: the result then agrees
// with swj_residual to the residual's rounding, not bit for bit.
//
// * The array is SWJ_NOALLOC_SCRATCH_BYTES (16 MiB) and lives on every GPU
//   that loads the library until the process exits.
// * Host code cannot use the array's name as a device address, so the first
//   call on each device looks its address up with cudaGetSymbolAddress (with
//   that device current) and caches it; that first call should come before
//   any stream capture.
// * Every call on a device shares the one array and leaves its contents
//   behind.  Every part of it a call reads was written earlier in the same
//   call, so nothing needs clearing, but calls whose work overlaps on the GPU
//   (other streams, other host threads) race on it: serialise them.
// * No cudaMalloc, cudaFree or allocating library routine is called.
#include "swj_internal.h"
#include <mutex>
#include <string.h>

__device__ __align__(256) unsigned char g_swj_noalloc_scratch[SWJ_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_na_mutex;
void *g_na_base[kMaxDevices];

int na_base(void **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return SWJ_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return SWJ_EINVAL;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_base[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_swj_noalloc_scratch) != cudaSuccess || !p) return SWJ_ECUDA;
        g_na_base[dev] = p;
    }
    *out = g_na_base[dev];
    return SWJ_OK;
}

// Forward-sweep coefficients of the spline system (same matrix as the
// context path builds on the host) and F, eps, written straight into the
// scratch.
__global__ void k_na_setup(int M, double *cp, double *a, double *inv, double *Fd, double *epsd,
                           double F, double eps)
{
    if (blockIdx.x || threadIdx.x) return;
    Fd[0] = F;
    epsd[0] = eps;
    cp[0] = 0.0; a[0] = 0.0; inv[0] = 1.0;
    for (int j = 1; j < M; ++j) {
        double aj = (j < M - 1) ? 1.0 : 2.0;
        double bj = (j < M - 1) ? 4.0 : 1.0;
        double cj = (j < M - 1) ? 1.0 : 0.0;
        double den = bj - aj * cp[j - 1];
        a[j] = aj;
        inv[j] = 1.0 / den;
        cp[j] = cj / den;
    }
}

inline long long na_round(long long bytes) { return (bytes + 255) & ~255LL; }

struct Carver {
    unsigned char *base;
    size_t off, cap;
    void *take(size_t bytes)
    {
        size_t o = off;
        off = (off + bytes + 255) & ~(size_t)255;
        return (off <= cap) ? base + o : nullptr;   // o is a multiple of 256
    }
};

}  // namespace

extern "C" int swj_residual_noalloc(const swj_mesh *mesh, double F, double eps, const double *u_dev,
                                    double *E_dev, int precision, void *stream)
{
    if (!mesh || !u_dev || !E_dev || u_dev == E_dev) return SWJ_EINVAL;
    if (!(mesh->N >= 4 && mesh->M >= 3 && mesh->dx > 0.0 && mesh->dy > 0.0 && mesh->n_rad >= 0.0))
        return SWJ_EINVAL;
    if (!(F > 0.0) || !(eps >= 0.0)) return SWJ_EINVAL;
    if (precision != SWJ_FP64 && precision != SWJ_FP32) return SWJ_EINVAL;
    const long long S = (long long)mesh->N * mesh->M, T = (long long)(mesh->N - 1) * mesh->M;
    // every piece the scratch holds, each rounded up to 256 bytes as the
    // carver takes it; the partial sums need at least one chunk (P = 1)
    const long long fixed = 4 * na_round(S * 8) + 3 * na_round((long long)mesh->M * 8) + 2 * na_round(T * 8) +
                            na_round(S * (long long)sizeof(SrcRec64)) + na_round(S * (long long)sizeof(SrcRec32)) +
                            na_round(8 * T * 8) + na_round(8 * T * 4) + 2 * na_round(8);
    if (fixed + na_round(T * 8) > (long long)SWJ_NOALLOC_SCRATCH_BYTES) return SWJ_ESIZE;

    void *base = nullptr;
    int rc = na_base(&base);
    if (rc) return rc;

    swj_ctx c;
    memset((void *)&c, 0, sizeof(c));
    c.mesh = *mesh;
    c.nb = 1;
    c.stream = (cudaStream_t)stream;
    if (cudaGetDevice(&c.dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, c.dev) != cudaSuccess)
        return SWJ_ECUDA;
    c.N = mesh->N;
    c.M = mesh->M;
    c.n1 = c.N + 1;
    c.H = c.n1 * c.M;
    c.nu = 2 * c.H;
    c.T = (int)T;
    c.S = (int)S;

    Carver cv{(unsigned char *)base, 0, (size_t)SWJ_NOALLOC_SCRATCH_BYTES};
    c.zeta = (double *)cv.take(S * 8);
    c.g = (double *)cv.take(S * 8);
    c.zetay = (double *)cv.take(S * 8);
    c.gy = (double *)cv.take(S * 8);
    c.spl_cp = (double *)cv.take((size_t)c.M * 8);
    c.spl_a = (double *)cv.take((size_t)c.M * 8);
    c.spl_inv = (double *)cv.take((size_t)c.M * 8);
    c.e2part = (double *)cv.take(T * 8);
    c.Ival = (double *)cv.take(T * 8);
    c.src64 = (SrcRec64 *)cv.take(S * sizeof(SrcRec64));
    c.src32 = (SrcRec32 *)cv.take(S * sizeof(SrcRec32));
    double *t64 = (double *)cv.take(8 * T * 8);
    float *t32 = (float *)cv.take(8 * T * 4);
    if (!t32) return SWJ_ESIZE;
    c.tgt64 = TgtArrays64{t64, t64 + T, t64 + 2 * T, t64 + 3 * T, t64 + 4 * T, t64 + 5 * T,
                                t64 + 6 * T, t64 + 7 * T};
    c.tgt32 = TgtArrays32{t32, t32 + T, t32 + 2 * T, t32 + 3 * T, t32 + 4 * T, t32 + 5 * T,
                          t32 + 6 * T, t32 + 7 * T};
    c.Fd = (double *)cv.take(8);
    c.epsd = (double *)cv.take(8);
    if (!c.epsd) return SWJ_ESIZE;
    // the launch plan of the context path, with fewer source chunks if the
    // partial sums would not fit the rest of the scratch (the pair sum is then
    // added in another order: the same value to rounding, not bit for bit)
    PairPlan pl = swj_pair_plan(&c, precision);
    long long maxP = (long long)(cv.cap - cv.off) / (T * 8);
    if (maxP < 1) return SWJ_ESIZE;
    if (pl.P > maxP) {
        pl.chunk = (int)((S + maxP - 1) / maxP);
        pl.P = (int)((S + pl.chunk - 1) / pl.chunk);
    }
    c.partial = (double *)cv.take((size_t)pl.P * T * 8);
    if (!c.partial) return SWJ_ESIZE;

    SWJ_COUNT_LAUNCH();
    k_na_setup<<<1, 1, 0, c.stream>>>(c.M, c.spl_cp, c.spl_a, c.spl_inv, c.Fd, c.epsd, F, eps);
    swj_launch_mesh_step(&c, u_dev, E_dev, nullptr);
    if (precision == SWJ_FP64) swj_launch_pairs64(&c, pl, nullptr);
    else swj_launch_pairs32(&c, pl, nullptr);
    swj_launch_assemble(&c, E_dev, pl.P, nullptr);
    SWJ_CUDA_TRY(cudaGetLastError());
    return SWJ_OK;
}
