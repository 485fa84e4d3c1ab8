// k_conv_tc.cu -- the 3x3x3 convolution of the learned block preconditioner
// on the 5th-generation tensor cores (tcgen05 + TMA, sm_103a).
//
//   out[v][co] = act(bias[co] + sum_tap sum_ci in[v + off(tap)][ci] W[tap][co][ci])
//
// activations channels-last [z][y][x][16] bf16, zero outside the grid;
// W [tap][co][ci] bf16 with tap = 9 (dz+1) + 3 (dy+1) + (dx+1); FP32
// accumulation; act = ReLU or identity.  As a GEMM per output tile: M = 128
// voxels (8 x 16 of one z-slice), N = 16 output channels, K = 27 taps x 16
// input channels, issued as 27 MMAs of K = 16 (kind::f16, bf16 operands,
// FP32 accumulator in tensor memory).
//
// Operand staging: a CTA walks a column of output tiles in z (work item = 8
// x 16 voxels x up to 16 slices) and keeps a ring of 4 halo planes (10 x 18
// voxels each, z-1 .. z+2) in shared memory; each tile loads only the next
// plane, one TMA load per 8-channel half (zero-filled outside the grid), as
// rows of 16 bytes, x fastest.  In the no-swizzle K-major layout a core
// matrix is 8 rows of 16 bytes, so the A operand of tap (dx, dy, dz) is the
// plane of z + dz seen from row (dy, dx): eight consecutive x of one y-row
// form a core matrix, the next y-row is 10 rows (160 bytes) further (the
// stride-dimension offset) and the second 8-channel half is the other
// half-plane (the leading-dimension offset).  No operand is copied per tap.
// Weights sit in shared memory in the same layout (per tap: 2 halves x 16
// rows x 16 bytes).
//
// Pipeline (persistent CTAs, 4 warps, 5 CTAs per SM): thread 0 issues the
// TMA load of the plane the next tile needs, waits for the current tile's
// planes, issues its 27 MMAs and commits them to an mbarrier; all four warps
// then read their 32 accumulator lanes (one voxel per thread, 16 columns),
// add the bias, apply the activation and store 32 bytes per voxel.  Every
// wait is bounded: on timeout the kernel raises a device error flag, waits
// (bounded) for its copies in flight, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstdint>

#include "perf_kernels.h"

namespace perf {

namespace {

constexpr int kCh = 16;
constexpr int kNTaps = 27;
constexpr int kTX = 8, kTY = 16;                   // output tile, one z-slice: M = 128
constexpr int kHX = kTX + 2, kHY = kTY + 2;         // its halo in x and y
constexpr int kPlaneRows = kHX * kHY;               // 180 rows of 16 bytes per half-plane
constexpr int kHalfBytes = kPlaneRows * 16;         // 2880
constexpr int kHalf = (kHalfBytes + 127) / 128 * 128;   // 2944: 128-byte aligned halves
constexpr int kPlaneBytes = 2 * kHalf;              // 5888: one z-plane of the halo
constexpr int kRing = 4;                            // planes z-1, z, z+1 and the next
constexpr int kZChunk = 16;                         // z-slices per work item
constexpr int kWBytes = kNTaps * 512;               // 13824
constexpr int kOffW = kRing * kPlaneBytes;          // 23552
constexpr int kOffBar = kOffW + kWBytes;            // 37376
constexpr int kSmemUsed = kOffBar + 64;             // full[4], mma, tmem address, abort flag
constexpr int kSmemDyn = kSmemUsed + 1024;          // room to align the base to 1024
constexpr int kTCThreads = 128;
constexpr int kCtasPerSm = 5;                       // 5 x 38.5 KB of shared memory
constexpr int kTmemCols = 32;                       // smallest allocation; 16 used
constexpr uint32_t kSpinLimit = 1u << 20;           // try_wait rounds before giving up

// M = 128, N = 16, bf16 x bf16 -> f32, both operands K-major.
constexpr uint32_t kIdesc = (1u << 4)                 // D format f32
                            | (1u << 7)               // A format bf16
                            | (1u << 10)              // B format bf16
                            | ((16u >> 3) << 17)      // N >> 3
                            | ((128u >> 4) << 24);    // M >> 4

__device__ int g_conv_tc_error;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

// Bounded wait for the phase with the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          uint32_t limit = kSpinLimit) {
    for (uint32_t i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (i >= 32) __nanosleep(128);
    }
    return false;
}

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int c0, int c1, int c2, int c3, int c4) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4),
        "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor, no swizzle: start address, leading-
// dimension (K direction) and stride-dimension (M/N direction) byte offsets
// between core matrices; bit 46 is the descriptor version of this family.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
           ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                        uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
}

struct Column {
    int x0, y0, z_lo, z_hi;
};

__device__ __forceinline__ Column item_coords(long long t, int nx, int ny, int G) {
    Column c;
    const long long pl = (long long)nx * ny;
    const int zc = (int)(t / pl);
    const int r = (int)(t - (long long)zc * pl);
    c.y0 = (r / nx) * kTY;
    c.x0 = (r % nx) * kTX;
    c.z_lo = zc * kZChunk;
    c.z_hi = min(c.z_lo + kZChunk, G);
    return c;
}

__device__ __forceinline__ int ring_slot(int q) { return (q + kRing) & (kRing - 1); }   // q >= -1

__global__ void __launch_bounds__(kTCThreads) k_conv_fwd_tc(const __grid_constant__ CUtensorMap in_map,
                                                            const __nv_bfloat16* __restrict__ W,
                                                            const float* __restrict__ bias,
                                                            __nv_bfloat16* __restrict__ out, int G,
                                                            int relu, uint32_t first_limit) {
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_addr(smem_raw);
    const uint32_t pad = (1024u - (raw & 1023u)) & 1023u;
    unsigned char* sm = smem_raw + pad;
    const uint32_t base = raw + pad;
    const uint32_t bar_full = base + kOffBar;   // + 8 slot
    const uint32_t bar_mma = base + kOffBar + 8 * kRing;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + kOffBar + 8 * kRing + 8);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + kOffBar + 8 * kRing + 12);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int q = 0; q < kRing; ++q) mbar_init(bar_full + 8 * q, 1);
        mbar_init(bar_mma, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // weights: B operand of tap t = planes [t][half][co][8 ci] (16 bytes a row)
    for (int i = threadIdx.x; i < kNTaps * kCh * 2; i += blockDim.x) {
        const int half = i & 1, co = (i >> 1) & (kCh - 1), tap = i >> 5;
        const __nv_bfloat16* src = W + (tap * kCh + co) * kCh + half * 8;
        uint4 v;
        if ((reinterpret_cast<uintptr_t>(src) & 15u) == 0) {
            v = *reinterpret_cast<const uint4*>(src);
        } else {
            uint32_t w4[4];
            for (int q = 0; q < 4; ++q)
                w4[q] = (uint32_t)__bfloat16_as_ushort(src[2 * q]) |
                        ((uint32_t)__bfloat16_as_ushort(src[2 * q + 1]) << 16);
            v = make_uint4(w4[0], w4[1], w4[2], w4[3]);
        }
        *reinterpret_cast<uint4*>(sm + kOffW + tap * 512 + half * 256 + co * 16) = v;
    }
    // the generic-proxy weight stores must be visible to the tensor cores
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const int nx = (G + kTX - 1) / kTX, ny = (G + kTY - 1) / kTY;
    const int nzc = (G + kZChunk - 1) / kZChunk;
    const long long n_items = (long long)nx * ny * nzc;
    float bs[kCh];
#pragma unroll
    for (int c = 0; c < kCh; ++c) bs[c] = bias ? bias[c] : 0.0f;

    // thread 0: loads issued into / waits completed on each ring slot
    int loaded[kRing], waited[kRing];
#pragma unroll
    for (int q = 0; q < kRing; ++q) loaded[q] = waited[q] = 0;
    // both 8-channel halves of halo plane q (z = q) of the column into its slot
    auto load_plane = [&](const Column& c, int q) {
        const int sl = ring_slot(q);
        const uint32_t dst = base + (uint32_t)(sl * kPlaneBytes);
        mbar_expect_tx(bar_full + 8 * sl, 2u * kHalfBytes);
        tma_load_5d(dst, &in_map, bar_full + 8 * sl, 0, 0, c.x0 - 1, c.y0 - 1, q);
        tma_load_5d(dst + kHalf, &in_map, bar_full + 8 * sl, 0, 1, c.x0 - 1, c.y0 - 1, q);
        ++loaded[sl];
    };
    // the CTA's first wait takes first_limit rounds (kSpinLimit except when a
    // test makes it run out); every later one kSpinLimit
    bool first_wait = true;
    auto wait_plane = [&](int q) -> bool {
        const int sl = ring_slot(q);
        const bool ok = mbar_wait(bar_full + 8 * sl, (uint32_t)waited[sl] & 1u,
                                  first_wait ? first_limit : kSpinLimit);
        first_wait = false;
        if (ok) ++waited[sl];
        return ok;
    };

    int it = 0;   // tiles processed by this CTA (phase of the MMA barrier)
    for (long long item = blockIdx.x; item < n_items && !*abort_flag; item += gridDim.x) {
        const Column c = item_coords(item, nx, ny, G);
        if (threadIdx.x == 0) {
            load_plane(c, c.z_lo - 1);
            load_plane(c, c.z_lo);
            load_plane(c, c.z_lo + 1);
        }
        for (int z = c.z_lo; z < c.z_hi; ++z, ++it) {
            bool ok = true;
            if (threadIdx.x == 0) {
                // plane z+2 serves the next tile; its slot held plane z-2,
                // last read by the previous tile's MMAs, which have completed
                if (z + 2 <= c.z_hi) load_plane(c, z + 2);
                if (z == c.z_lo) ok = wait_plane(z - 1) && wait_plane(z);
                ok = ok && wait_plane(z + 1);
                if (ok) {
                    tc_fence_after();
                    // descriptors: constant high words; per tap only the start address moves
                    const uint64_t a_hi = smem_desc(0u, kHalf, kHX * 16);
                    const uint64_t b0 = smem_desc(base + kOffW, 256, 128);
                    uint32_t pl[3];
#pragma unroll
                    for (int hz = 0; hz < 3; ++hz)
                        pl[hz] = base + (uint32_t)(ring_slot(z - 1 + hz) * kPlaneBytes);
#pragma unroll
                    for (int tap = 0; tap < kNTaps; ++tap) {
                        const int hx = tap % 3, hy = (tap / 3) % 3, hz = tap / 9;
                        const uint64_t a = a_hi | (uint64_t)(((pl[hz] + (uint32_t)((hy * kHX + hx) * 16)) &
                                                              0x3FFFFu) >> 4);
                        mma_f16(tmem, a, b0 + (uint64_t)(tap * 32), tap > 0 ? 1u : 0u);
                    }
                    mma_commit(bar_mma);
                } else {
                    atomicExch(&g_conv_tc_error, 1);
                    *abort_flag = 1;
                }
            }
            __syncwarp();
            if (threadIdx.x != 0 || ok) ok = mbar_wait(bar_mma, (uint32_t)it & 1u);
            if (!ok) {
                atomicExch(&g_conv_tc_error, 1);
                *abort_flag = 1;
            }
            // tcgen05.ld is warp-collective: the whole warp reads or none of it
            ok = __all_sync(0xffffffffu, ok);
            if (ok) {
                tc_fence_after();
                uint32_t r[16];
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16), r);
                const int m = warp * 32 + lane;
                const int x = c.x0 + (m & (kTX - 1)), y = c.y0 + (m >> 3);
                if (x < G && y < G) {
                    float o[kCh];
#pragma unroll
                    for (int q = 0; q < kCh; ++q) {
                        o[q] = __uint_as_float(r[q]) + bs[q];
                        if (relu) o[q] = fmaxf(o[q], 0.0f);
                    }
                    uint4* dst = reinterpret_cast<uint4*>(out + (((long long)z * G + y) * G + x) * kCh);
                    dst[0] = make_uint4(pack2(o[0], o[1]), pack2(o[2], o[3]), pack2(o[4], o[5]),
                                        pack2(o[6], o[7]));
                    dst[1] = make_uint4(pack2(o[8], o[9]), pack2(o[10], o[11]), pack2(o[12], o[13]),
                                        pack2(o[14], o[15]));
                }
            }
            tc_fence_before();
            __syncthreads();
            if (*abort_flag) break;
        }
    }
    // error path: loads still in flight land before the CTA exits
    if (threadIdx.x == 0) {
        for (int q = 0; q < kRing; ++q)
            while (waited[q] < loaded[q]) {
                if (!mbar_wait(bar_full + 8 * q, (uint32_t)waited[q] & 1u)) break;
                ++waited[q];
            }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols)
                     : "memory");
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Rounds of the first TMA wait of each CTA (see lpc_conv_set_first_wait_limit).
uint32_t g_first_wait_limit = kSpinLimit;

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

}  // namespace

cudaError_t lpc_conv_fwd(const __nv_bfloat16* in, const __nv_bfloat16* W, const float* bias,
                         __nv_bfloat16* out, int G, int relu, cudaStream_t st) {
    if (G <= 0) return cudaSuccess;
    if ((reinterpret_cast<uintptr_t>(in) & 15u) || (reinterpret_cast<uintptr_t>(out) & 15u))
        return cudaErrorMisalignedAddress;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    // in as (8 channels, 2 halves, x, y, z): byte strides of dims 1..4
    const cuuint64_t dims[5] = {8, 2, (cuuint64_t)G, (cuuint64_t)G, (cuuint64_t)G};
    const cuuint64_t strides[4] = {16, 32, 32ull * G, 32ull * G * G};
    const cuuint32_t box[5] = {8, 1, kHX, kHY, 1};   // one z-plane of a column's halo
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    CUtensorMap map;
    const CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<__nv_bfloat16*>(in),
                           dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    // per call: the current device may differ between calls
    cudaError_t e = cudaFuncSetAttribute(k_conv_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSmemDyn);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (sms <= 0) sms = 1;
    const long long nx = (G + kTX - 1) / kTX, ny = (G + kTY - 1) / kTY;
    const long long items = nx * ny * ((G + kZChunk - 1) / kZChunk);
    const long long cap = (long long)sms * kCtasPerSm;
    const int grid = (int)(items < cap ? items : cap);
    k_conv_fwd_tc<<<grid, kTCThreads, kSmemDyn, st>>>(map, W, bias, out, G, relu,
                                                      g_first_wait_limit);
    count_launch();
    return cudaGetLastError();
}

// Test hook: the number of polling rounds of each CTA's first wait for its
// TMA loads in later launches (0 makes that wait give up at once, so the
// timeout path -- raise the flag, drain the loads in flight with the normal
// limit, free tensor memory, return -- runs without any fault); values above
// the normal limit are clamped to it.
void lpc_conv_set_first_wait_limit(uint32_t rounds) {
    g_first_wait_limit = rounds < kSpinLimit ? rounds : kSpinLimit;
}

// Reads and clears the device flag raised by a convolution whose bounded
// waits ran out (1), else 0.  Synchronises with the device.
int lpc_conv_error() {
    int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_conv_tc_error, sizeof(int)) != cudaSuccess) return -1;
    if (v) {
        const int z = 0;
        cudaMemcpyToSymbol(g_conv_tc_error, &z, sizeof(int));
    }
    return v;
}

}  // namespace perf
