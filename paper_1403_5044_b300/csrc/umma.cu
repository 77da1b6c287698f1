// The digit-slice products of the band LU's sliced block products (Ozaki's
// splitting, see ozaki.cu) on the fifth-generation tensor cores: tcgen05.mma
// with bf16 operands staged in shared memory by TMA and FP32 accumulators in
// tensor memory.
//
// For block product t (A = slices of slot a, B = slices of slot b, s digits of
// beta bits each) and output o of the digit scheme (level d, digits p0..p1;
// OzScheme) the kernel forms
//     T_o = sum_{p=p0..p1} a_p b_(d-p)        (np x np, FP32)
// (the outputs of level d together make T_d = sum_{p=0..d} a_p b_(d-p)).
// Both operands are stored K-major with the same shape [slot][row][digit][np]:
// row r of A holds a_0[r, :] .. a_(s-1)[r, :]; row c of B holds column c of
// b_0 .. b_(s-1).  T_o[r, c] is then the dot product of A's row r over digits
// p0..p1 with B's row c over digits d-p0..d-p1, so the zero products a_p b_q
// with p + q > d are never formed.  Every partial sum is an integer below
// 2^24 (beta and the outputs' length are chosen for that), so FP32
// accumulation is exact in any order and the result equals any other exact
// evaluation bit for bit.
//
// One CTA per output tile (t, o, 128-row tile, tn-column tile): M = 128 x
// N = tn x K = 16 MMAs, tn = np split into equal parts of at most 192, rounded
// up to 16 (TMA fills rows and columns past np with zeros); K runs over digit
// p and 64-element chunks of it.  Warp 0 lane 0 issues the
// TMA loads into a two-stage ring (81 KB of shared memory, 256 tensor-memory
// columns: two CTAs per SM, so one CTA's prologue and epilogue overlap the
// other's MMAs), warp 1 lane 0 issues the MMAs (one
// tcgen05.commit frees each stage), warp 2 owns the tensor-memory allocation,
// and all four warps read the accumulator back (tcgen05.ld, one warp per 32
// rows) and store the np x np tile of T_o.  Tiles run longest output first.
// Every mbarrier wait is bounded: a wait that runs out sets *err and
// the CTA skips the rest of its work, still waiting (bounded) for its own TMA
// loads and MMAs in flight before it frees its tensor memory and exits.
#include "swj_internal.h"
#include <cuda.h>
#include <map>
#include <mutex>
#include <tuple>

namespace {

constexpr int kTM = 128, kTN = 192, kTK = 64, kStages = 2, kThreads = 128;
constexpr int kABytes = kTM * kTK * 2;            // one stage of A: 128 rows x 128 B
constexpr int kBBytes = kTN * kTK * 2;            // room for B: up to 192 rows x 128 B
constexpr int kStageBytes = kABytes + kBBytes;
constexpr int kSmemBytes = kStages * kStageBytes + 1024;   // + alignment of the ring to 1024 B
constexpr uint32_t kTmemCols = 256;               // >= kTN FP32 columns, a power of two
constexpr long long kWaitLimit = 1ll << 24;       // mbarrier try_wait rounds (each may suspend)

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *mb, int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(mb)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *mb, int bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(mb)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *mb, int parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(su32(mb)), "r"(parity) : "memory");
    return ok != 0;
}

// bounded wait for the phase of the given parity to complete
__device__ __forceinline__ bool mbar_wait(uint64_t *mb, int parity)
{
    for (long long it = 0; it < kWaitLimit; ++it)
        if (mbar_try(mb, parity)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, uint64_t *mb, int x, int y, int z,
                                            int w)
{
    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4, %5}], [%6];"
                 ::"r"(su32(dst)), "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(w), "r"(su32(mb))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major operand tile written by TMA
// with the 128-byte swizzle: rows of 128 B (64 bf16), 8-row atoms of 1024 B
// stacked along M (N) at a stride of 1024 B; the leading-dimension offset is
// unused for this layout.  Fields: start address >> 4 (bits 0-13), leading
// byte offset >> 4 (16-29), stride byte offset >> 4 (32-45), the descriptor
// version 1 (46-48), base offset 0 (the ring is 1024-byte aligned), swizzle
// mode 2 = 128 B (61-63).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), bf16
// A and B (7-9 = 1, 10-12 = 1), both K-major (15, 16 = 0), N >> 3 (17-22),
// M >> 4 (24-28).
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "setp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
                 : "memory");
}

// arrive on the mbarrier once every tcgen05 operation this thread issued so far has completed
__device__ __forceinline__ void umma_commit(uint64_t *mb)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(mb))
                 : "memory");
}

// 32 lanes x 16 consecutive FP32 columns of tensor memory, lane i of the warp
// reading TMEM lane (taddr >> 16) + i
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32"
                 " {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                   "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(kThreads, 2)
k_oz_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
          const OzProd *__restrict__ prods, int count, const __grid_constant__ OzScheme z, int tn, int mtiles,
          int ntiles, int kch, float *__restrict__ P, int *err)
{
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages], accb;
    __shared__ uint32_t tmem_slot;
    __shared__ int bad;
    unsigned char *ring = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // tile order: the longest outputs first (z.order), then t, row tile, column tile
    const int per = count * mtiles * ntiles, np = z.np;
    const int oi = z.order[(int)blockIdx.x / per];
    const int d = z.d[oi], p0 = z.p0[oi];
    const int rem = (int)blockIdx.x % per;
    const int t = rem / (mtiles * ntiles), mt = (rem / ntiles) % mtiles, nt = rem % ntiles;
    const int nk = kch * (z.p1[oi] - p0 + 1);   // K chunks: digits p = p0..p1, kch 64-element chunks each
    const int stage_tx = kABytes + tn * kTK * 2;
    if (threadIdx.x == 0) {
        for (int i = 0; i < kStages; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        mbar_init(&accb, 1);
        bad = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const OzProd o = prods[t];

    if (warp == 0 && lane == 0) {
        // producer: stage kc % kStages takes chunk kc once the MMAs of chunk kc - kStages are done
        asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&tmA) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&tmB) : "memory");
        int issued = 0;
        for (int kc = 0; kc < nk; ++kc) {
            const int st = kc % kStages;
            if (kc >= kStages && !mbar_wait(&empty[st], ((kc / kStages) - 1) & 1)) {
                bad = 1;
                atomicExch(err, 1);
                break;
            }
            if (*(volatile int *)&bad) break;
            unsigned char *sa = ring + (size_t)st * kStageBytes, *sb = sa + kABytes;
            const int pp = kc / kch, jc = kc - kch * pp, p = p0 + pp;
            mbar_expect_tx(&full[st], stage_tx);
            tma_load_4d(sa, &tmA, &full[st], kTK * jc, p, kTM * mt, o.a);
            tma_load_4d(sb, &tmB, &full[st], kTK * jc, d - p, tn * nt, o.b);
            issued = kc + 1;
        }
        // loads still in flight (only after a failed wait): let them land before the exit
        for (int kc = (issued > kStages ? issued - kStages : 0); kc < issued; ++kc)
            mbar_wait(&full[kc % kStages], (kc / kStages) & 1);
    } else if (warp == 1 && lane == 0) {
        const uint32_t ring_s = su32(ring), idesc = idesc_bf16(kTM, tn);
        for (int kc = 0; kc < nk; ++kc) {
            const int st = kc % kStages;
            if (!mbar_wait(&full[st], (kc / kStages) & 1)) {
                bad = 1;
                atomicExch(err, 1);
                break;
            }
            tc_fence_after();
            const uint32_t a0 = ring_s + (uint32_t)(st * kStageBytes), b0 = a0 + kABytes;
#pragma unroll
            for (int k = 0; k < kTK / 16; ++k)   // K = 16 bf16 = 32 B per MMA inside the 128-B swizzle atom
                umma_bf16(tmem, sw128_desc(a0 + 32 * k), sw128_desc(b0 + 32 * k), idesc, (kc | k) != 0);
            umma_commit(&empty[st]);
        }
        umma_commit(&accb);   // also after a failure: the wait below then covers every MMA in flight
    }
    __syncwarp();
    const bool ok = mbar_wait(&accb, 0);
    tc_fence_after();
    if (ok && !*(volatile int *)&bad) {
        const int r = kTM * mt + 32 * warp + lane, cb = tn * nt, ce = min(np, cb + tn);
        float *row = P + ((size_t)(t * z.nout + oi) * np + r) * np;
        const uint32_t tl = tmem + ((uint32_t)(32 * warp) << 16);
        for (int c0 = cb; c0 < ce; c0 += 16) {
            float v[16];
            tmem_ld16(tl + (uint32_t)(c0 - cb), v);   // every lane of the warp takes part
            if (r < np) {
                const int nc = min(16, ce - c0);   // np and tn are multiples of 8
                float4 *dst = (float4 *)(row + c0);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (4 * q < nc) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            }
        }
    } else if (threadIdx.x == 0 && !ok) {
        atomicExch(err, 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 2) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

std::mutex g_map_mutex;
std::map<std::tuple<const void *, int, int, size_t, int>, CUtensorMap> g_maps;

// 4-D map of slices [slot][row][digit][np] (bf16), box {64, 1, rows_box, 1},
// 128-byte swizzle, zeros outside the tensor; cached per buffer and shape
int slice_map(CUtensorMap *out, const void *base, int np, int s, size_t nslots, int rows_box)
{
    std::lock_guard<std::mutex> lock(g_map_mutex);
    auto key = std::make_tuple(base, np, s, nslots, rows_box);
    auto it = g_maps.find(key);
    if (it != g_maps.end()) {
        *out = it->second;
        return SWJ_OK;
    }
    static EncodeTiledFn encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return SWJ_ECUDA;
        encode = (EncodeTiledFn)fn;
    }
    const cuuint64_t dims[4] = {(cuuint64_t)np, (cuuint64_t)s, (cuuint64_t)np, (cuuint64_t)nslots};
    const cuuint64_t strides[3] = {(cuuint64_t)np * 2, (cuuint64_t)s * np * 2, (cuuint64_t)np * s * np * 2};
    const cuuint32_t box[4] = {(cuuint32_t)kTK, 1, (cuuint32_t)rows_box, 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    CUtensorMap m;
    if (encode(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return SWJ_ECUDA;
    g_maps[key] = m;
    *out = m;
    return SWJ_OK;
}

}  // namespace

int swj_oz_gemm(cudaStream_t st, const OzScheme &z, int count, const OzProd *prods, const void *sa, size_t nsa,
                const void *sb, size_t nsb, float *P, int *err)
{
    if (count <= 0) return SWJ_OK;
    const int np = z.np, s = z.s;
    if (z.nout < 1 || z.nout > kOzMaxOut) return SWJ_EINVAL;
    // np a multiple of 8 (16-byte digit rows for TMA), 16-byte aligned slices
    if (np < 8 || np % 8 || s < 1 || ((uintptr_t)sa | (uintptr_t)sb) % 16) return SWJ_EINVAL;
    const int ntiles = (np + kTN - 1) / kTN;
    const int tn = ((np + ntiles - 1) / ntiles + 15) / 16 * 16;   // <= 192, a multiple of 16
    const int mtiles = (np + kTM - 1) / kTM, kch = (np + kTK - 1) / kTK;
    CUtensorMap mA, mB;
    int rc = slice_map(&mA, sa, np, s, nsa, kTM);
    if (rc) return rc;
    if ((rc = slice_map(&mB, sb, np, s, nsb, tn))) return rc;
    static bool attr = false;
    if (!attr) {
        SWJ_CUDA_TRY(cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes));
        attr = true;
    }
    SWJ_COUNT_LAUNCH();
    k_oz_gemm<<<count * z.nout * mtiles * ntiles, kThreads, kSmemBytes, st>>>(mA, mB, prods, count, z, tn, mtiles,
                                                                              ntiles, kch, P, err);
    SWJ_CUDA_TRY(cudaGetLastError());
    return SWJ_OK;
}
