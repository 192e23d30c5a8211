// tcgen05 tensor-core path of the block contraction (K-b..K-f fused, K-i).
//
// Same decomposition as the FP32 path: rows are meson rows (A = conj(phi_i))
// and diquark rows (A = phi_i x phi_j, i<j, colex order), columns are (k,p)
// with Psi = ph_p(x) phi_k, and the complex product runs over K = 3V
// (site, colour):  C[row][col] = sum A(x,c) Psi(x,c).
//
// Complex -> real embedding (no extra flops): A is interleaved (re, im) along
// K; every complex column becomes two real B rows,
//   re-row [Psi_re, -Psi_im]  ->  C_re,    im-row [Psi_im, Psi_re]  ->  C_im.
//
// Precision: phi is rescaled by an exact power of two per timeslice; every
// operand value v is split into hi = RN16(v), lo = RN16(v - hi) (FP16 or
// BF16); the tensor core accumulates hi*hi + hi*lo + lo*hi (hi*hi only in the
// plain modes) in FP32.  The tensor core's FP32 accumulation does not round
// to nearest, so its error grows with the number of additions; the
// accumulator is therefore drained every `chunk_stages` K stages into a
// second tensor-memory region of FP32 running sums kept by CUDA cores with
// round-to-nearest, and at the end of a tile the sums are scaled back and
// written to the complex128 output in FP64.
//
// Tile: 128 rows x 96 complex columns (UMMA M = 128, N = 192), K stage = 32
// complex entries (one 128-byte swizzled row of FP16 per operand row).
// Tensor memory (512 columns): ACC [0,192) | SUM [192,384) | A slots 2 x 64.
// Shared memory: NB B stages (hi+lo, 48 KB each) and 2 staging buffers that
// hold, per stage, the 12-site windows of every vector the tile's rows use
// and the phases of those sites.
//
// Warp roles (512 threads, persistent CTAs, static tile order):
//   0-3   A producers: thread = tile row = TMEM lane; reads its vectors'
//         windows from the staging buffer, forms the 32 K entries of the
//         stage (diquark or conj(phi)), splits and tcgen05.st's them;
//   4-9   B producers: (column, 4-entry K group) units; phi_k from global
//         memory with coalesced loads, phase from the staging buffer;
//         writes hi/lo words in the 128B-swizzled K-major layout;
//   10-13 epilogue: drains ACC into SUM, writes the output at tile end;
//   14    loader: cp.async of the staging windows, completion on an mbarrier;
//   15    TMEM allocation and single-thread MMA issue.
// Every wait on an mbarrier is bounded; on expiry the CTA records
// STATUS_TIMEOUT, raises a shared abort flag and all roles return.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "laph_internal.cuh"

namespace laph {
namespace {

constexpr int NTHREADS = 512;
constexpr int WARP_B0 = 4;
constexpr int N_BWARPS = 6;
constexpr int WARP_E0 = 10;
constexpr int WARP_LOAD = 14;
constexpr int WARP_MMA = 15;
constexpr int KSTAGE = 32;                    // complex K entries per stage (= 64 real)
constexpr int B_ROWS = 2 * TC_TC;             // real B rows per tile (192)
constexpr int B_BYTES = B_ROWS * 128;         // one of hi/lo
constexpr int STAGE_BYTES = 2 * B_BYTES;      // hi + lo
constexpr int WIN_SITES = 14;                 // staged sites per stage (from the even site <= x0)
constexpr int WIN = 3 * WIN_SITES;            // staged complex entries per vector
constexpr int VEC_STRIDE = WIN * 8;           // 336 B = 84 words: LDS.128 of 8 consecutive slots hit distinct banks
constexpr int PH_STRIDE = WIN_SITES * 8;      // 112 B = 28 words, likewise
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t ACC_COL = 0;
constexpr uint32_t SUM_COL = 192;
constexpr uint32_t A_COL = 384;
constexpr uint32_t A_SLOT_COLS = 64;          // 32 columns hi + 32 columns lo
constexpr long long WAIT_LIMIT = 4000000000LL; // cycles (about 2 s at the top clock)

static_assert(TC_TR == 128 && TC_TC == 96, "layout assumes 128 x 96 tiles");
static_assert(A_COL + 2 * A_SLOT_COLS == TMEM_COLS, "tensor memory budget");

struct Shared {
    uint64_t stg_full[3], stg_empty[3];
    uint64_t a_full[2], a_empty[2];
    uint64_t b_full[3], b_empty[3];
    uint64_t acc_full, acc_empty;
    uint64_t done;
    uint32_t tmem_base;
    int abort;
};

// ------------------------------------------------------------ PTX wrappers

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Waits up to about `hint_ns` for the phase with the given parity to
// complete; the warp is suspended meanwhile instead of spinning.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity, uint32_t hint_ns = 20000u)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Bulk global -> shared copy (16-byte aligned addresses, size a multiple of
// 16) whose completion is counted in bytes on the mbarrier.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[tmem] * B[smem]^T, kind::f16, FP32 accumulate.
__device__ __forceinline__ void mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                       uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

#define LAPH_R32(v)                                                                                              \
    "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]), \
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]),          \
        "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]),           \
        "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
#define LAPH_W32(v)                                                                                              \
    "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),  \
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),   \
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),  \
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
        LAPH_R32(v)
        : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : LAPH_W32(v)
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), version 1.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(16u >> 4) << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor, kind::f16: FP32 D, FP16 (0) or BF16 (1) A and B,
// both K-major, M = 128, N = n_real.
__device__ __forceinline__ uint32_t idesc_f16(int n_real, int bf16)
{
    return (1u << 4) | ((uint32_t)bf16 << 7) | ((uint32_t)bf16 << 10) | ((uint32_t)(n_real >> 3) << 17) |
           ((uint32_t)(128 >> 4) << 24);
}

// Byte offset of 16-byte chunk j (0..7) of real row n in a 128B-swizzled,
// K-major operand whose rows are 128 bytes.
__device__ __forceinline__ uint32_t swz(int n, int j) { return (uint32_t)((n >> 3) * 1024 + (n & 7) * 128 + ((j ^ (n & 7)) << 4)); }

// ------------------------------------------------------------ numerics

// hi = RN(a), lo = RN(a - hi) for a pair (a -> low half, b -> high half).
template <int ELEM>
__device__ __forceinline__ void split2(float a, float b, uint32_t &hi, uint32_t &lo)
{
    if (ELEM == 0) {
        const __half2 h = __floats2half2_rn(a, b);
        const float2 hf = __half22float2(h);
        const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    } else {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    }
}

// Power-of-two exponent s with max|phi| * 2^s in [0.5, 1).
__device__ __forceinline__ int scale_exp(unsigned maxbits)
{
    if (maxbits == 0) return 0;
    int E = (int)((maxbits >> 23) & 0xff);
    if (E == 0) E = 1;
    int s = 126 - E;
    return s > 100 ? 100 : (s < -100 ? -100 : s);
}
__device__ __forceinline__ float pow2f(int s) { return __int_as_float((127 + s) << 23); }
__device__ __forceinline__ double pow2d(int s) { return __longlong_as_double((long long)(1023 + s) << 52); }

// ------------------------------------------------------------ waits

struct Ctx {
    Shared *S;
    int *status;
    int lane;
};

// Warp-wide bounded wait (every lane calls it; the result is warp-uniform).
// Each try_wait suspends the warp until the phase completes or about 20 us
// pass; between those wake-ups the abort flag and the time limit are checked.
__device__ __forceinline__ bool warp_wait(const Ctx &c, uint64_t *bar, uint32_t parity)
{
    if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;
    const long long t0 = clock64();
    while (true) {
        if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;
        const int ab = *(volatile int *)&c.S->abort;
        if (__any_sync(0xffffffffu, ab != 0)) return false;
        int expired = (clock64() - t0) > WAIT_LIMIT;
        expired = __shfl_sync(0xffffffffu, expired, 0);
        if (expired) {
            if (c.lane == 0) {
                *(volatile int *)&c.S->abort = 1;
                atomicOr(c.status, STATUS_TIMEOUT);
            }
            return false;
        }
    }
}

// ------------------------------------------------------------ A producer

// Staged windows hold WIN_SITES sites starting at the even site x0e <= x0
// (x0 = first site of the stage).  OFF = kappa0 - 3*x0e in [0, 5] is the
// window position of the stage's first K entry, so K entry kl of the stage is
// window entry kl + OFF.

// Pair row: the stage's K entries from the windows of phi_i (wi) and phi_j
// (wj), read two sites (three 16-byte loads) at a time.
template <int ELEM, int OFF>
__device__ __forceinline__ void a_pair(const float2 *wi, const float2 *wj, float sc2, uint32_t (&hi)[32],
                                       uint32_t (&lo)[32])
{
#pragma unroll
    for (int m = 0; m < WIN_SITES / 2; m++) {
        if (6 * m - OFF > KSTAGE - 1) break;
        if (6 * m + 5 - OFF < 0) continue;
        float2 u[6], v[6];
#pragma unroll
        for (int h = 0; h < 3; h++) {
            const float4 a = *reinterpret_cast<const float4 *>(wi + 6 * m + 2 * h);
            const float4 b = *reinterpret_cast<const float4 *>(wj + 6 * m + 2 * h);
            u[2 * h] = make_float2(a.x, a.y);
            u[2 * h + 1] = make_float2(a.z, a.w);
            v[2 * h] = make_float2(b.x, b.y);
            v[2 * h + 1] = make_float2(b.z, b.w);
        }
#pragma unroll
        for (int s = 0; s < 2; s++) {
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const int kl = 3 * (2 * m + s) + c - OFF;
                if (kl < 0 || kl >= KSTAGE) continue;
                const float2 d = cross_c(u + 3 * s, v + 3 * s, c);
                split2<ELEM>(d.x * sc2, d.y * sc2, hi[kl], lo[kl]);
            }
        }
    }
}

// Meson row: conj(phi_i) at window entries kl + OFF.
template <int ELEM, int OFF>
__device__ __forceinline__ void a_meson(const float2 *wi, float sc, uint32_t (&hi)[32], uint32_t (&lo)[32])
{
#pragma unroll
    for (int f = OFF / 2; f <= (OFF + KSTAGE - 1) / 2; f++) {
        const float4 a = *reinterpret_cast<const float4 *>(wi + 2 * f);
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int kl = 2 * f + h - OFF;
            if (kl < 0 || kl >= KSTAGE) continue;
            const float re = h ? a.z : a.x, im = h ? a.w : a.y;
            split2<ELEM>(re * sc, -im * sc, hi[kl], lo[kl]);
        }
    }
}

template <int ELEM, int OFF>
__device__ __forceinline__ void produce_a_off(int kind, const float2 *wi, const float2 *wj, float sc,
                                              uint32_t (&hi)[32], uint32_t (&lo)[32])
{
    if (kind == 2)
        a_pair<ELEM, OFF>(wi, wj, sc * sc, hi, lo);
    else if (kind == 1)
        a_meson<ELEM, OFF>(wi, sc, hi, lo);
    else {
#pragma unroll
        for (int kl = 0; kl < KSTAGE; kl++) hi[kl] = lo[kl] = 0u;
    }
}

template <int ELEM>
__device__ __forceinline__ void produce_a(int kind, int off, const float2 *wi, const float2 *wj, float sc,
                                          uint32_t (&hi)[32], uint32_t (&lo)[32])
{
    switch (off) {
    case 0: produce_a_off<ELEM, 0>(kind, wi, wj, sc, hi, lo); break;
    case 1: produce_a_off<ELEM, 1>(kind, wi, wj, sc, hi, lo); break;
    case 2: produce_a_off<ELEM, 2>(kind, wi, wj, sc, hi, lo); break;
    case 3: produce_a_off<ELEM, 3>(kind, wi, wj, sc, hi, lo); break;
    case 4: produce_a_off<ELEM, 4>(kind, wi, wj, sc, hi, lo); break;
    default: produce_a_off<ELEM, 5>(kind, wi, wj, sc, hi, lo); break;
    }
}

// ------------------------------------------------------------ the kernel

struct KParams {
    const InstDev *insts;
    const TileDev *tiles;
    const unsigned *maxbits;
    int *status;
    int n_tiles;
    int chunk_stages;
    int stg_bytes;   // bytes of one staging buffer
    int ph_off;      // offset of the phase rows inside a staging buffer
    int nb;          // B stage buffers (2 or 3)
    int nstg;        // staging buffers (2 or 3)
    int debug_stall;
};

template <int ELEM, int TERMS>
__global__ void __launch_bounds__(NTHREADS, 1) tc_kernel(const KParams kp)
{
    extern __shared__ uint8_t smem_raw[];
    // align to 1024 bytes by offsetting the __shared__ array itself, so that
    // the compiler keeps every derived pointer in the shared address space
    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint8_t *bstage = smem;
    uint8_t *stage_buf = smem + kp.nb * STAGE_BYTES;
    Shared *S = reinterpret_cast<Shared *>(stage_buf + kp.nstg * kp.stg_bytes);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int NB = kp.nb, NS = kp.nstg;
    Ctx c{S, kp.status, lane};

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; s++) {
            mbar_init(&S->stg_full[s], 1);
            mbar_init(&S->stg_empty[s], 4 + N_BWARPS);
        }
        for (int s = 0; s < 2; s++) {
            mbar_init(&S->a_full[s], 4);
            mbar_init(&S->a_empty[s], 1);
        }
        for (int s = 0; s < NB; s++) {
            mbar_init(&S->b_full[s], N_BWARPS);
            mbar_init(&S->b_empty[s], 1);
        }
        mbar_init(&S->acc_full, 1);
        mbar_init(&S->acc_empty, 4);
        mbar_init(&S->done, 1);
        S->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == WARP_MMA) {
        tmem_alloc(&S->tmem_base, TMEM_COLS);
        tmem_relinquish();
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S->tmem_base;

    if (warp == WARP_LOAD) {
        // ---------------------------------------------------------- loader
        uint32_t g = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < kp.n_tiles && ok; tile += gridDim.x) {
            const TileDev td = kp.tiles[tile];
            const InstDev &I = kp.insts[td.inst];
            const long long Vs = I.Vs;
            const int K = (int)(3 * I.V);
            const int P = I.P;
            const float2 *phit = I.phi_tc + (long long)td.t * I.N * Vs * 3;
            const int n_st = (K + KSTAGE - 1) / KSTAGE;
            const int nsl = td.nv + td.nk;
            for (int st = 0; st < n_st; st++, g++) {
                const int buf = g % NS;
                if (!warp_wait(c, &S->stg_empty[buf], ((g / NS) & 1u) ^ 1u)) {
                    ok = false;
                    break;
                }
                uint8_t *base = stage_buf + buf * kp.stg_bytes;
                const long long x0e = (long long)((st * KSTAGE) / 3) & ~1LL;
                const int nsite = (int)((Vs - x0e) < WIN_SITES ? (Vs - x0e) : WIN_SITES);  // even
                const uint32_t vbytes = 24u * nsite, pbytes = 8u * nsite;
                if (lane == 0) mbar_arrive_expect_tx(&S->stg_full[buf], vbytes * nsl + pbytes * P);
                __syncwarp();
                for (int idx = lane; idx < nsl + P; idx += 32) {
                    if (idx < nsl) {
                        const int vec = idx < td.nv ? td.v_lo + idx : td.k_lo + (idx - td.nv);
                        bulk_g2s(base + idx * VEC_STRIDE, phit + ((long long)vec * Vs + x0e) * 3, vbytes,
                                 &S->stg_full[buf]);
                    } else {
                        const int p = idx - nsl;
                        bulk_g2s(base + kp.ph_off + p * PH_STRIDE, I.phase + (long long)p * Vs + x0e, pbytes,
                                 &S->stg_full[buf]);
                    }
                }
            }
        }
    } else if (warp < WARP_B0) {
        // ---------------------------------------------------------- A producers
        const int quad = warp & 3;
        const int r = quad * 32 + lane;
        const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
        uint32_t g = 0;
        bool stalled = false, ok = true;
        for (int tile = blockIdx.x; tile < kp.n_tiles && ok; tile += gridDim.x) {
            const TileDev td = kp.tiles[tile];
            const InstDev &I = kp.insts[td.inst];
            const int K = (int)(3 * I.V);
            const int gr = td.row0 + r;
            int kind = 0, vi = 0, vj = 0;
            if (gr < I.rows) {
                if (gr < I.mes_rows) {
                    kind = 1;
                    vi = gr;
                } else {
                    kind = 2;
                    pair_of(gr - I.mes_rows, vi, vj);
                }
            }
            const int si = kind ? vi - td.v_lo : 0, sj = kind == 2 ? vj - td.v_lo : 0;
            const float sc = pow2f(scale_exp(kp.maxbits[I.ts_base + td.t]));
            const int n_st = (K + KSTAGE - 1) / KSTAGE;
            for (int st = 0; st < n_st; st++, g++) {
                const int sa = g & 1;
                const int buf = g % NS;
                if (!warp_wait(c, &S->a_empty[sa], ((g >> 1) & 1u) ^ 1u) ||
                    !warp_wait(c, &S->stg_full[buf], (g / NS) & 1u)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const int kap0 = st * KSTAGE;
                const int off = kap0 - 3 * (((kap0 / 3)) & ~1);
                const uint8_t *base = stage_buf + buf * kp.stg_bytes;
                const float2 *wi = reinterpret_cast<const float2 *>(base + si * VEC_STRIDE);
                const float2 *wj = reinterpret_cast<const float2 *>(base + sj * VEC_STRIDE);
                uint32_t hi[32], lo[32];
                produce_a<ELEM>(kind, off, wi, wj, sc, hi, lo);
                __syncwarp();
                if (lane == 0) mbar_arrive(&S->stg_empty[buf]);
                if (kap0 + KSTAGE > K) {  // last stage of the tile: entries past 3V are zero
#pragma unroll
                    for (int kl = 0; kl < KSTAGE; kl++)
                        if (kap0 + kl >= K) hi[kl] = lo[kl] = 0u;
                }
                const uint32_t ta = tmem + lane_base + A_COL + (uint32_t)sa * A_SLOT_COLS;
                tmem_st32(ta, hi);
                tmem_st32(ta + 32, lo);
                tmem_wait_st();
                tc_fence_before();
                __syncwarp();
                const bool skip = kp.debug_stall && !stalled && blockIdx.x == 0 && warp == 0;
                if (skip) stalled = true;
                if (lane == 0 && !skip) mbar_arrive(&S->a_full[sa]);
            }
        }
    } else if (warp < WARP_E0) {
        // ---------------------------------------------------------- B producers
        const int tb = (warp - WARP_B0) * 32 + lane;  // 0..191
        uint32_t g = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < kp.n_tiles && ok; tile += gridDim.x) {
            const TileDev td = kp.tiles[tile];
            const InstDev &I = kp.insts[td.inst];
            const int K = (int)(3 * I.V);
            const int P = I.P;
            const int ncols = td.ncols;
            const int ncols_pad = (ncols + 7) & ~7;
            const float sc = pow2f(scale_exp(kp.maxbits[I.ts_base + td.t]));
            // four units per thread: unit u = tb + 192 m -> column cu = u / 8, K group q = u % 8
            int kslot[4], pp[4], cu[4], qq[4];
            bool valid[4], write[4];
#pragma unroll
            for (int m = 0; m < 4; m++) {
                const int u = tb + 192 * m;
                cu[m] = u >> 3;
                qq[m] = u & 7;
                valid[m] = cu[m] < ncols;
                write[m] = cu[m] < ncols_pad;
                int k = td.k_lo, p = 0;
                if (valid[m]) {
                    k = (td.col0 + cu[m]) / P;
                    p = td.col0 + cu[m] - k * P;
                }
                kslot[m] = td.nv + (k - td.k_lo);
                pp[m] = p;
            }
            const int n_st = (K + KSTAGE - 1) / KSTAGE;
            for (int st = 0; st < n_st; st++, g++) {
                const int sb = g % NB;
                const int buf = g % NS;
                if (!warp_wait(c, &S->b_empty[sb], ((g / NB) & 1u) ^ 1u) ||
                    !warp_wait(c, &S->stg_full[buf], (g / NS) & 1u)) {
                    ok = false;
                    break;
                }
                const int kap0 = st * KSTAGE;
                const int off = kap0 - 3 * (((kap0 / 3)) & ~1);
                const uint8_t *base = stage_buf + buf * kp.stg_bytes;
                uint8_t *bhi = bstage + sb * STAGE_BYTES;
                uint8_t *blo = bhi + B_BYTES;
#pragma unroll
                for (int m = 0; m < 4; m++) {
                    if (!write[m]) continue;
                    const float2 *wk = reinterpret_cast<const float2 *>(base + kslot[m] * VEC_STRIDE);
                    const float2 *wp = reinterpret_cast<const float2 *>(base + kp.ph_off + pp[m] * PH_STRIDE);
                    const int e0 = 4 * qq[m] + off;  // window entry of this group's first K entry
                    uint32_t rh[4], rl[4], ih[4], il[4];
#pragma unroll
                    for (int v = 0; v < 4; v++) {
                        const int e = e0 + v;
                        float2 psi = make_float2(0.f, 0.f);
                        if (valid[m] && kap0 + 4 * qq[m] + v < K) psi = cmulf(wp[e / 3], wk[e]);
                        uint32_t h, l;
                        split2<ELEM>(psi.x * sc, psi.y * sc, h, l);
                        rh[v] = h ^ 0x80000000u;            // (re, -im)
                        rl[v] = l ^ 0x80000000u;
                        ih[v] = __byte_perm(h, 0, 0x1032);  // (im, re)
                        il[v] = __byte_perm(l, 0, 0x1032);
                    }
                    const int n0 = 2 * cu[m];
                    *reinterpret_cast<uint4 *>(bhi + swz(n0, qq[m])) = make_uint4(rh[0], rh[1], rh[2], rh[3]);
                    *reinterpret_cast<uint4 *>(bhi + swz(n0 + 1, qq[m])) = make_uint4(ih[0], ih[1], ih[2], ih[3]);
                    *reinterpret_cast<uint4 *>(blo + swz(n0, qq[m])) = make_uint4(rl[0], rl[1], rl[2], rl[3]);
                    *reinterpret_cast<uint4 *>(blo + swz(n0 + 1, qq[m])) = make_uint4(il[0], il[1], il[2], il[3]);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&S->stg_empty[buf]);
                fence_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&S->b_full[sb]);
            }
        }
    } else if (warp < WARP_LOAD) {
        // ---------------------------------------------------------- epilogue
        const int quad = warp & 3;
        const int r = quad * 32 + lane;
        const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
        uint32_t gc = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < kp.n_tiles && ok; tile += gridDim.x) {
            const TileDev td = kp.tiles[tile];
            const InstDev &I = kp.insts[td.inst];
            const int K = (int)(3 * I.V);
            const int ncols = td.ncols;
            const int n_real = 2 * ((ncols + 7) & ~7);
            const int gr = td.row0 + r;
            const bool rvalid = gr < I.rows;
            const bool meson = gr < I.mes_rows;
            int pj = 0;
            long long q = 0;
            if (rvalid && !meson) {
                int pi_;
                q = gr - I.mes_rows;
                pair_of(q, pi_, pj);
            }
            const int s = scale_exp(kp.maxbits[I.ts_base + td.t]);
            const double fac = meson ? pow2d(-2 * s) : pow2d(-3 * s);
            const int n_st = (K + KSTAGE - 1) / KSTAGE;
            const int n_ch = (n_st + kp.chunk_stages - 1) / kp.chunk_stages;
            for (int ch = 0; ch < n_ch; ch++, gc++) {
                if (!warp_wait(c, &S->acc_full, gc & 1u)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                for (int b = 0; b * 32 < n_real; b++) {
                    uint32_t va[32], vs[32];
                    tmem_ld32(tmem + lane_base + ACC_COL + 32u * b, va);
                    if (ch > 0) tmem_ld32(tmem + lane_base + SUM_COL + 32u * b, vs);
                    tmem_wait_ld();
                    if (ch > 0) {
#pragma unroll
                        for (int e = 0; e < 32; e++)
                            va[e] = __float_as_uint(__uint_as_float(va[e]) + __uint_as_float(vs[e]));
                    }
                    tmem_st32(tmem + lane_base + SUM_COL + 32u * b, va);
                }
                tmem_wait_st();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&S->acc_empty);
            }
            if (!ok) break;
            // tile done: FP32 sums -> FP64 output, scale undone
            const long long tP = (long long)td.t * I.P;
            for (int b = 0; b * 32 < n_real; b++) {
                uint32_t v[32];
                tmem_ld32(tmem + lane_base + SUM_COL + 32u * b, v);
                tmem_wait_ld();
#pragma unroll
                for (int u = 0; u < 16; u++) {
                    const int cc = 16 * b + u;
                    if (!rvalid || cc >= ncols) continue;
                    const int col = td.col0 + cc;
                    const int k = col / I.P, p = col - k * I.P;
                    double2 *dst;
                    if (meson) {
                        dst = I.outM + ((tP + p) * I.N + gr) * I.N + k;
                    } else {
                        if (k <= pj) continue;
                        dst = I.outB + (tP + p) * I.n_trip + binom3(k) + q;
                    }
                    *dst = make_double2((double)__uint_as_float(v[2 * u]) * fac,
                                        (double)__uint_as_float(v[2 * u + 1]) * fac);
                }
            }
        }
    } else {
        // ---------------------------------------------------------- MMA issue
        uint32_t g = 0, gc = 0;
        bool issued = false, ok = true;
        for (int tile = blockIdx.x; tile < kp.n_tiles && ok; tile += gridDim.x) {
            const TileDev td = kp.tiles[tile];
            const InstDev &I = kp.insts[td.inst];
            const int K = (int)(3 * I.V);
            const int n_real = 2 * ((td.ncols + 7) & ~7);
            const uint32_t idesc = idesc_f16(n_real, ELEM);
            const int n_st = (K + KSTAGE - 1) / KSTAGE;
            for (int st = 0; st < n_st; st++, g++) {
                const bool chunk_start = (st % kp.chunk_stages) == 0;
                const bool chunk_end = ((st + 1) % kp.chunk_stages) == 0 || st + 1 == n_st;
                if (chunk_start && !warp_wait(c, &S->acc_empty, (gc & 1u) ^ 1u)) {
                    ok = false;
                    break;
                }
                const int sa = g & 1, sb = g % NB;
                if (!warp_wait(c, &S->a_full[sa], (g >> 1) & 1u) || !warp_wait(c, &S->b_full[sb], (g / NB) & 1u)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                if (lane == 0) {
                    const uint32_t a_hi = tmem + A_COL + (uint32_t)sa * A_SLOT_COLS, a_lo = a_hi + 32;
                    const uint32_t b_hi = smem_u32(bstage + sb * STAGE_BYTES), b_lo = b_hi + B_BYTES;
                    const uint32_t d = tmem + ACC_COL;
#pragma unroll
                    for (int ks = 0; ks < 4; ks++) {
                        const uint32_t acc = (chunk_start && ks == 0) ? 0u : 1u;
                        mma_ts(d, a_hi + 8 * ks, desc_sw128(b_hi + 32 * ks), idesc, acc);
                        if (TERMS == 3) {
                            mma_ts(d, a_hi + 8 * ks, desc_sw128(b_lo + 32 * ks), idesc, 1u);
                            mma_ts(d, a_lo + 8 * ks, desc_sw128(b_hi + 32 * ks), idesc, 1u);
                        }
                    }
                    mma_commit(&S->a_empty[sa]);
                    mma_commit(&S->b_empty[sb]);
                    if (chunk_end) mma_commit(&S->acc_full);
                    issued = true;
                }
                __syncwarp();
                if (chunk_end) gc++;
            }
        }
        // every issued MMA has completed before tensor memory is released
        if (lane == 0 && issued) mma_commit(&S->done);
        __syncwarp();
        if (__shfl_sync(0xffffffffu, issued ? 1 : 0, 0)) warp_wait(c, &S->done, 0u);
    }

    __syncthreads();
    if (warp == WARP_MMA) {
        tc_fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
}

int stg_bytes_for(int max_staged, int max_P)
{
    const int b = max_staged * VEC_STRIDE + max_P * PH_STRIDE;
    return (b + 127) & ~127;
}

int smem_for(int nb, int nstg, int stg_bytes) { return nb * STAGE_BYTES + nstg * stg_bytes + (int)sizeof(Shared) + 1024; }

constexpr int SMEM_LIMIT = 227 * 1024;

template <int ELEM, int TERMS>
cudaError_t launch_one(const InstDev *d_inst, const TileDev *d_tiles, long long n_tiles, const unsigned *maxbits,
                       const TcConfig &cfg, int *status, cudaStream_t s)
{
    KParams kp;
    kp.insts = d_inst;
    kp.tiles = d_tiles;
    kp.maxbits = maxbits;
    kp.status = status;
    kp.n_tiles = (int)n_tiles;
    kp.chunk_stages = (cfg.chunk_sites * 3) / KSTAGE;
    if (kp.chunk_stages < 1) kp.chunk_stages = 1;
    kp.stg_bytes = stg_bytes_for(cfg.max_staged, cfg.max_P);
    kp.ph_off = cfg.max_staged * VEC_STRIDE;
    kp.debug_stall = cfg.debug_stall;
    // deepest buffering that fits: staging 3 then B stages 3
    const int choices[4][2] = {{3, 3}, {2, 3}, {3, 2}, {2, 2}};
    int smem = 0;
    kp.nb = 0;
    for (int ch = 0; ch < 4; ch++) {
        const int need = smem_for(choices[ch][0], choices[ch][1], kp.stg_bytes);
        if (need <= SMEM_LIMIT) {
            kp.nb = choices[ch][0];
            kp.nstg = choices[ch][1];
            smem = need;
            break;
        }
    }
    if (!kp.nb) return cudaErrorNotSupported;
    cudaError_t e = cudaFuncSetAttribute(tc_kernel<ELEM, TERMS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int grid = cfg.grid > 0 ? cfg.grid : 148;
    if ((long long)grid > n_tiles) grid = (int)n_tiles;
    tc_kernel<ELEM, TERMS><<<grid, NTHREADS, smem, s>>>(kp);
    return cudaGetLastError();
}

}  // namespace

int tc_smem_bytes() { return smem_for(2, 2, stg_bytes_for(TC_MAX_STAGED, TC_MAX_P)); }

cudaError_t launch_tc(const InstDev *d_inst, const TileDev *d_tiles, long long n_tiles, const unsigned *d_maxbits,
                      unsigned long long *d_counter, const TcConfig &cfg, int *d_status, cudaStream_t s)
{
    (void)d_counter;
    if (n_tiles <= 0) return cudaSuccess;
    if (n_tiles > 0x7fffffffLL || cfg.max_staged > TC_MAX_STAGED || cfg.max_P > TC_MAX_P) return cudaErrorNotSupported;
    if (cfg.elem == 0 && cfg.terms == 3) return launch_one<0, 3>(d_inst, d_tiles, n_tiles, d_maxbits, cfg, d_status, s);
    if (cfg.elem == 1 && cfg.terms == 3) return launch_one<1, 3>(d_inst, d_tiles, n_tiles, d_maxbits, cfg, d_status, s);
    if (cfg.elem == 0 && cfg.terms == 1) return launch_one<0, 1>(d_inst, d_tiles, n_tiles, d_maxbits, cfg, d_status, s);
    if (cfg.elem == 1 && cfg.terms == 1) return launch_one<1, 1>(d_inst, d_tiles, n_tiles, d_maxbits, cfg, d_status, s);
    return cudaErrorNotSupported;
}

}  // namespace laph
