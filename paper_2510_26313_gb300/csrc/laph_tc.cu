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
// Precision: the operands are built from a copy of phi rescaled by an exact
// power of two per timeslice; every operand value v is split into
// hi = RN16(v), lo = RN16(v - hi) (FP16 or BF16); the tensor core
// accumulates hi*hi + hi*lo + lo*hi (hi*hi only in the plain modes) in FP32.
// Its FP32 accumulation does not round to nearest, so its error grows with
// the number of additions; the accumulator is drained every `chunk_stages`
// K stages into a second tensor-memory region of FP32 running sums kept by
// CUDA cores with round-to-nearest, and at the end of a tile the sums are
// scaled back and written to the complex128 output in FP64.
//
// Tile: 128 rows x 96 complex columns (UMMA M = 128, N = 192), K stage = 32
// complex entries (one 128-byte swizzled row of FP16 per operand row).
// Tensor memory (512 columns): ACC [0,192) | SUM [192,384) | A slots 2 x 64.
// Shared memory: NB B stages (hi+lo, 48 KB each) and a ring of NR site-block
// buffers, each holding, for one block of TC_BS sites, the block slots of the
// tile's row vectors, of its column vectors and the block's phase rows --
// three bulk copies from the site-blocked, pre-scaled copy of phi.
//
// Warp roles (704 threads, persistent CTAs, static tile order):
//   0-7   A producers: two warps per TMEM lane quadrant, each forms 16 of the
//         stage's 32 K entries of its row (diquark or conj(phi)), splits and
//         tcgen05.st's them;
//   8-15  B producers: (column, 4-entry K group) units; Psi from the block
//         buffers; hi/lo words in the 128B-swizzled K-major layout;
//   16-19 epilogue: drains ACC into SUM, writes the output at tile end;
//   20    loader: bulk copies of the site blocks, completion on mbarriers;
//   21    TMEM allocation and single-thread MMA issue.
// Every wait on an mbarrier is bounded; on expiry the CTA records
// STATUS_TIMEOUT, raises a shared abort flag and all roles return.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "laph_internal.cuh"

namespace laph {
namespace {

constexpr int NTHREADS = 704;
constexpr int WARP_B0 = 8;
constexpr int N_AWARPS = 8;
constexpr int N_BWARPS = 8;
constexpr int B_UNITS = 3;                    // (column, K group) units per B producer thread: 96 x 8 / 256
constexpr int WARP_E0 = 16;
constexpr int WARP_LOAD = 20;
constexpr int WARP_MMA = 21;
constexpr int KSTAGE = 32;                    // complex K entries per stage (= 64 real)
constexpr int KHALF = 16;                     // K entries per A producer warp per stage
constexpr int B_ROWS = 2 * TC_TC;             // real B rows per tile (192)
constexpr int B_BYTES = B_ROWS * 128;         // one of hi/lo
constexpr int STAGE_BYTES = 2 * B_BYTES;      // hi + lo
constexpr int SLOT_BYTES = TC_SLOT * 8;       // 208 B = 52 words: LDS.128 of 8 consecutive slots hit distinct banks
constexpr int PHROW_BYTES = TC_PHROW * 8;     // 88 B = 22 words: LDS.64 of 16 consecutive rows hit distinct banks
constexpr int MAX_NB = 3, MAX_NR = 6;
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t ACC_COL = 0;
constexpr uint32_t SUM_COL = 192;
constexpr uint32_t A_COL = 384;
constexpr uint32_t A_SLOT_COLS = 64;          // 32 columns hi + 32 columns lo
constexpr long long WAIT_LIMIT = 4000000000LL; // cycles (about 2 s at the top clock)

static_assert(TC_TR == 128 && TC_TC == 96, "layout assumes 128 x 96 tiles");
static_assert(TC_BS == 8, "block arithmetic assumes 8-site blocks");
static_assert(A_COL + 2 * A_SLOT_COLS == TMEM_COLS, "tensor memory budget");

struct Shared {
    uint64_t blk_full[MAX_NR], blk_empty[MAX_NR];
    uint64_t a_full[2], a_empty[2];
    uint64_t b_full[MAX_NB], b_empty[MAX_NB];
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

__device__ __forceinline__ void tmem_st2(uint32_t taddr, uint32_t v0, uint32_t v1)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};" ::"r"(taddr), "r"(v0), "r"(v1) : "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
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
__device__ __noinline__ bool warp_wait(const Ctx &c, uint64_t *bar, uint32_t parity)
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

// ------------------------------------------------------------ site blocks

// Which site blocks of the current tile a warp has waited for / released.
// Every consumer warp waits for and releases every block of a tile in order,
// so that the ring's phases stay consistent.
struct BlockTrack {
    uint32_t gbase;  // global index of the tile's first block
    int waited, released;
};

__device__ __noinline__ bool wait_blocks(const Ctx &c, BlockTrack &tr, int upto, int NR)
{
    while (tr.waited < upto) {
        const uint32_t g = tr.gbase + tr.waited;
        if (!warp_wait(c, &c.S->blk_full[g % NR], (g / NR) & 1u)) return false;
        tr.waited++;
    }
    return true;
}

__device__ __noinline__ void release_blocks(const Ctx &c, BlockTrack &tr, int upto, int NR)
{
    if (upto > tr.waited) upto = tr.waited;
    if (tr.released < upto) {
        __syncwarp();
        while (tr.released < upto) {
            const uint32_t g = tr.gbase + tr.released;
            if (c.lane == 0) mbar_arrive(&c.S->blk_empty[g % NR]);
            tr.released++;
        }
    }
}

// ------------------------------------------------------------ A producer

// Component c of the colour cross product u x v as eight fused operations.
__device__ __forceinline__ float2 cross8(const float2 *u, const float2 *v, int c)
{
    const int a = (c + 1) % 3, b = (c + 2) % 3;
    float re = u[a].x * v[b].x;
    re = fmaf(-u[a].y, v[b].y, re);
    re = fmaf(-u[b].x, v[a].x, re);
    re = fmaf(u[b].y, v[a].y, re);
    float im = u[a].x * v[b].y;
    im = fmaf(u[a].y, v[b].x, im);
    im = fmaf(-u[b].x, v[a].y, im);
    im = fmaf(-u[b].y, v[a].x, im);
    return make_float2(re, im);
}

// The 16 K entries [ks, ks+16) of a stage for one row, written straight to
// tensor memory (hi at ta, lo at ta + 32).  Site pairs (2 sites = 6 K entries
// = three 16-byte loads per vector) pf..pf+3 cover the entries, pf = ks / 6;
// ks is even, so every pair's entries fall into whole column pairs that are
// either all inside [0, 16) or all outside.  The loop is kept rolled so that
// its code stays small.  kind: 2 diquark row, 1 meson row (conj(phi_i)), 0
// no row (loads suppressed, zeros written).
template <int ELEM>
__device__ __forceinline__ void a_half(int kind, int ks, const uint8_t *base0, const uint8_t *base1, int b0,
                                       int nblk, int si, int sj, uint32_t ta)
{
    const int pf = ks / 6;
#pragma unroll 1
    for (int m = 0; m < 4; m++) {
        const int kl0 = 6 * (pf + m) - ks;          // entry index of the pair's first K entry (even)
        if (kl0 >= KHALF) break;
        const int xg = 2 * (pf + m);                // first site of the pair
        const int b = xg >> 3;
        const bool in = b < nblk && kind != 0;
        const uint8_t *base = ((b == b0) ? base0 : base1) + (xg & 7) * 24;
        const float4 *wi = reinterpret_cast<const float4 *>(base + si * SLOT_BYTES);
        const float4 *wj = reinterpret_cast<const float4 *>(base + sj * SLOT_BYTES);
        float2 u[6], v[6];
#pragma unroll
        for (int h = 0; h < 3; h++) {
            const float4 a = in ? wi[h] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 bb = in ? wj[h] : make_float4(0.f, 0.f, 0.f, 0.f);
            u[2 * h] = make_float2(a.x, a.y);
            u[2 * h + 1] = make_float2(a.z, a.w);
            v[2 * h] = make_float2(bb.x, bb.y);
            v[2 * h + 1] = make_float2(bb.z, bb.w);
        }
#pragma unroll
        for (int e = 0; e < 6; e += 2) {
            const int kl = kl0 + e;
            if (kl < 0 || kl >= KHALF) continue;    // uniform over the warp
            uint32_t h0, l0, h1, l1;
#pragma unroll
            for (int f = 0; f < 2; f++) {
                const int q = e + f;
                const float2 dq = cross8(u + 3 * (q / 3), v + 3 * (q / 3), q % 3);
                const float2 d = kind == 2 ? dq : make_float2(u[q].x, -u[q].y);   // diquark or conj(phi_i)
                if (f == 0)
                    split2<ELEM>(d.x, d.y, h0, l0);
                else
                    split2<ELEM>(d.x, d.y, h1, l1);
            }
            tmem_st2(ta + kl, h0, h1);
            tmem_st2(ta + 32 + kl, l0, l1);
        }
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
    int blk_bytes;   // bytes of one site-block buffer
    int ph_off;      // offset of the phase rows inside a block buffer
    int nb;          // B stage buffers
    int nr;          // site-block buffers
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
    uint8_t *bbuf = smem + kp.nb * STAGE_BYTES;
    Shared *S = reinterpret_cast<Shared *>(bbuf + kp.nr * kp.blk_bytes);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int NB = kp.nb, NR = kp.nr;
    Ctx c{S, kp.status, lane};

    if (threadIdx.x == 0) {
        for (int s = 0; s < NR; s++) {
            mbar_init(&S->blk_full[s], 1);
            mbar_init(&S->blk_empty[s], N_AWARPS + N_BWARPS);
        }
        for (int s = 0; s < 2; s++) {
            mbar_init(&S->a_full[s], N_AWARPS);
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
        uint32_t gb = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < kp.n_tiles && ok; tile += gridDim.x) {
            const TileDev td = kp.tiles[tile];
            const InstDev &I = kp.insts[td.inst];
            const uint32_t bytesA = td.nv * SLOT_BYTES, bytesB = td.nk * SLOT_BYTES;
            const uint32_t bytesP = (uint32_t)I.phb_stride * 8u;
            for (int b = 0; b < I.nblk; b++) {
                const uint32_t g = gb + b;
                const int slot = g % NR;
                if (!warp_wait(c, &S->blk_empty[slot], ((g / NR) & 1u) ^ 1u)) {
                    ok = false;
                    break;
                }
                if (lane == 0) {
                    uint8_t *base = bbuf + slot * kp.blk_bytes;
                    const float2 *blk = I.phi_blk + ((long long)td.t * I.nblk + b) * I.N * TC_SLOT;
                    mbar_arrive_expect_tx(&S->blk_full[slot], bytesA + bytesB + bytesP);
                    bulk_g2s(base, blk + (long long)td.v_lo * TC_SLOT, bytesA, &S->blk_full[slot]);
                    bulk_g2s(base + bytesA, blk + (long long)td.k_lo * TC_SLOT, bytesB, &S->blk_full[slot]);
                    bulk_g2s(base + kp.ph_off, I.phase_blk + (long long)b * I.phb_stride, bytesP, &S->blk_full[slot]);
                }
                __syncwarp();
            }
            gb += I.nblk;
        }
    } else if (warp < WARP_B0) {
        // ---------------------------------------------------------- A producers
        const int quad = warp & 3, half = warp >> 2;
        const int r = quad * 32 + lane;
        const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
        uint32_t g = 0, gb = 0;
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
            const int nblk = I.nblk;
            BlockTrack tr{gb, 0, 0};
            const int n_st = (K + KSTAGE - 1) / KSTAGE;
            for (int st = 0; st < n_st; st++, g++) {
                const int sa = g & 1;
                const int ks = st * KSTAGE + KHALF * half;
                const int pf = ks / 6;
                const int bneed = min(nblk - 1, (2 * pf + 7) >> 3);
                if (!warp_wait(c, &S->a_empty[sa], ((g >> 1) & 1u) ^ 1u) || !wait_blocks(c, tr, bneed + 1, NR)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                // buffers of the (at most two) site blocks this half stage reads
                const int b0 = (2 * pf) >> 3;
                const int r0 = (int)((tr.gbase + b0) % NR);
                const uint8_t *base0 = bbuf + r0 * kp.blk_bytes;
                const uint8_t *base1 = bbuf + (r0 + 1 == NR ? 0 : r0 + 1) * kp.blk_bytes;
                const uint32_t ta = tmem + lane_base + A_COL + (uint32_t)sa * A_SLOT_COLS + KHALF * half;
                a_half<ELEM>(kind, ks, base0, base1, b0, nblk, si, sj, ta);
                // blocks the next stage does not need (sites before its first) are free
                release_blocks(c, tr, (((st + 1) * KSTAGE) / 3) >> 3, NR);
                tmem_wait_st();
                tc_fence_before();
                __syncwarp();
                const bool skip = kp.debug_stall && !stalled && blockIdx.x == 0 && warp == 0;
                if (skip) stalled = true;
                if (lane == 0 && !skip) mbar_arrive(&S->a_full[sa]);
            }
            if (ok && wait_blocks(c, tr, nblk, NR)) release_blocks(c, tr, nblk, NR);
            gb += nblk;
        }
    } else if (warp < WARP_E0) {
        // ---------------------------------------------------------- B producers
        const int tb = (warp - WARP_B0) * 32 + lane;  // 0..255
        uint32_t g = 0, gb = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < kp.n_tiles && ok; tile += gridDim.x) {
            const TileDev td = kp.tiles[tile];
            const InstDev &I = kp.insts[td.inst];
            const int K = (int)(3 * I.V);
            const int P = I.P;
            const int ncols = td.ncols;
            const int ncols_pad = (ncols + 7) & ~7;
            const int nblk = I.nblk;
            // B_UNITS units per thread: unit u = tb + 256 m -> column cu = u / 8, K group q = u % 8
            int koff[B_UNITS], poff[B_UNITS], cu[B_UNITS], qq[B_UNITS];
            bool valid[B_UNITS], write[B_UNITS];
#pragma unroll
            for (int m = 0; m < B_UNITS; m++) {
                const int u = tb + 256 * m;
                cu[m] = u >> 3;
                qq[m] = u & 7;
                valid[m] = cu[m] < ncols;
                write[m] = cu[m] < ncols_pad;
                int k = td.k_lo, p = 0;
                if (valid[m]) {
                    k = (td.col0 + cu[m]) / P;
                    p = td.col0 + cu[m] - k * P;
                }
                koff[m] = (td.nv + (k - td.k_lo)) * SLOT_BYTES;
                poff[m] = kp.ph_off + p * PHROW_BYTES;
            }
            BlockTrack tr{gb, 0, 0};
            const int n_st = (K + KSTAGE - 1) / KSTAGE;
            for (int st = 0; st < n_st; st++, g++) {
                const int sb = g % NB;
                const int kap0 = st * KSTAGE;
                const int bneed = min(nblk - 1, ((kap0 + KSTAGE - 1) / 3) >> 3);
                if (!warp_wait(c, &S->b_empty[sb], ((g / NB) & 1u) ^ 1u) || !wait_blocks(c, tr, bneed + 1, NR)) {
                    ok = false;
                    break;
                }
                // buffers of the (at most three) site blocks of this stage; block b
                // holds K entries [24 b, 24 b + 24)
                const int b0 = kap0 / 24;
                const int r0 = (int)((tr.gbase + b0) % NR);
                const int r1 = r0 + 1 == NR ? 0 : r0 + 1;
                const int r2 = r1 + 1 == NR ? 0 : r1 + 1;
                const uint8_t *base0 = bbuf + r0 * kp.blk_bytes, *base1 = bbuf + r1 * kp.blk_bytes,
                              *base2 = bbuf + r2 * kp.blk_bytes;
                uint8_t *bhi = bstage + sb * STAGE_BYTES;
                uint8_t *blo = bhi + B_BYTES;
#pragma unroll 1
                for (int m = 0; m < B_UNITS; m++) {
                    if (!write[m]) continue;
                    const int k4 = kap0 + 4 * qq[m];
                    const int rb = k4 / 24 - b0;        // block of the first entry, relative to b0
                    int e = k4 - 24 * (b0 + rb);        // entry within the block: 3 * site + colour
                    const uint8_t *base = rb == 0 ? base0 : (rb == 1 ? base1 : base2);
                    const uint8_t *nbase = rb == 0 ? base1 : base2;   // next block, if the group crosses
                    int cc = e % 3;
                    const uint8_t *pf_ = base + koff[m] + e * 8;          // phi_k entry
                    const uint8_t *pp_ = base + poff[m] + (e / 3) * 8;    // phase of its site
                    uint32_t rh[4], rl[4], ih[4], il[4];
#pragma unroll
                    for (int v = 0; v < 4; v++) {
                        float2 psi = make_float2(0.f, 0.f);
                        if (valid[m] && k4 + v < K)
                            psi = cmulf(*reinterpret_cast<const float2 *>(pp_), *reinterpret_cast<const float2 *>(pf_));
                        uint32_t h, l;
                        split2<ELEM>(psi.x, psi.y, h, l);
                        rh[v] = h ^ 0x80000000u;            // (re, -im)
                        rl[v] = l ^ 0x80000000u;
                        ih[v] = __byte_perm(h, 0, 0x1032);  // (im, re)
                        il[v] = __byte_perm(l, 0, 0x1032);
                        pf_ += 8;
                        if (++cc == 3) {
                            cc = 0;
                            pp_ += 8;
                        }
                        if (++e == 3 * TC_BS) {             // next site block
                            e = 0;
                            pf_ = nbase + koff[m];
                            pp_ = nbase + poff[m];
                        }
                    }
                    const int n0 = 2 * cu[m];
                    *reinterpret_cast<uint4 *>(bhi + swz(n0, qq[m])) = make_uint4(rh[0], rh[1], rh[2], rh[3]);
                    *reinterpret_cast<uint4 *>(bhi + swz(n0 + 1, qq[m])) = make_uint4(ih[0], ih[1], ih[2], ih[3]);
                    *reinterpret_cast<uint4 *>(blo + swz(n0, qq[m])) = make_uint4(rl[0], rl[1], rl[2], rl[3]);
                    *reinterpret_cast<uint4 *>(blo + swz(n0 + 1, qq[m])) = make_uint4(il[0], il[1], il[2], il[3]);
                }
                release_blocks(c, tr, (((st + 1) * KSTAGE) / 3) >> 3, NR);
                fence_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&S->b_full[sb]);
            }
            if (ok && wait_blocks(c, tr, nblk, NR)) release_blocks(c, tr, nblk, NR);
            gb += nblk;
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
                for (int b = 0; b * 16 < n_real; b++) {
                    uint32_t va[16], vs[16];
                    tmem_ld16(tmem + lane_base + ACC_COL + 16u * b, va);
                    if (ch > 0) tmem_ld16(tmem + lane_base + SUM_COL + 16u * b, vs);
                    tmem_wait_ld();
                    if (ch > 0) {
#pragma unroll
                        for (int e = 0; e < 16; e++)
                            va[e] = __float_as_uint(__uint_as_float(va[e]) + __uint_as_float(vs[e]));
                    }
                    tmem_st16(tmem + lane_base + SUM_COL + 16u * b, va);
                }
                tmem_wait_st();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&S->acc_empty);
            }
            if (!ok) break;
            // tile done: FP32 sums -> FP64 output, scale undone
            const long long tP = (long long)td.t * I.P;
            for (int b = 0; b * 16 < n_real; b++) {
                uint32_t v[16];
                tmem_ld16(tmem + lane_base + SUM_COL + 16u * b, v);
                tmem_wait_ld();
#pragma unroll 1
                for (int u = 0; u < 8; u++) {
                    const int cc = 8 * b + u;
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
                    // descriptor start addresses advance 32 bytes (2 units of 16) per K step
                    const uint64_t dhi = desc_sw128(smem_u32(bstage + sb * STAGE_BYTES));
                    const uint64_t dlo = dhi + (uint64_t)(B_BYTES >> 4);
                    const uint32_t d = tmem + ACC_COL;
#pragma unroll
                    for (int ks = 0; ks < 4; ks++) {
                        const uint32_t acc = (chunk_start && ks == 0) ? 0u : 1u;
                        mma_ts(d, a_hi + 8 * ks, dhi + 2 * ks, idesc, acc);
                        if (TERMS == 3) {
                            mma_ts(d, a_hi + 8 * ks, dlo + 2 * ks, idesc, 1u);
                            mma_ts(d, a_lo + 8 * ks, dhi + 2 * ks, idesc, 1u);
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

int blk_bytes_for(int max_staged, int max_phb)
{
    const int b = max_staged * SLOT_BYTES + max_phb * 8;
    return (b + 127) & ~127;
}

int smem_for(int nb, int nr, int blk_bytes) { return nb * STAGE_BYTES + nr * blk_bytes + (int)sizeof(Shared) + 1024; }

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
    kp.blk_bytes = blk_bytes_for(cfg.max_staged, cfg.max_phb);
    kp.ph_off = cfg.max_staged * SLOT_BYTES;
    kp.debug_stall = cfg.debug_stall;
    // deepest buffering that fits (a stage reads up to three site blocks)
    const int choices[5][2] = {{3, 6}, {3, 5}, {3, 4}, {2, 5}, {2, 4}};
    int smem = 0;
    kp.nb = 0;
    for (int ch = 0; ch < 5; ch++) {
        const int need = smem_for(choices[ch][0], choices[ch][1], kp.blk_bytes);
        if (need <= SMEM_LIMIT) {
            kp.nb = choices[ch][0];
            kp.nr = choices[ch][1];
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

int tc_smem_bytes() { return smem_for(2, 4, blk_bytes_for(TC_MAX_STAGED, ((TC_MAX_P * TC_PHROW * 8 + 15) / 16) * 2)); }

cudaError_t launch_tc(const InstDev *d_inst, const TileDev *d_tiles, long long n_tiles, const unsigned *d_maxbits,
                      unsigned long long *d_counter, const TcConfig &cfg, int *d_status, cudaStream_t s)
{
    (void)d_counter;
    if (n_tiles <= 0) return cudaSuccess;
    if (n_tiles > 0x7fffffffLL || cfg.max_staged > TC_MAX_STAGED) return cudaErrorNotSupported;
    if (cfg.elem == 0 && cfg.terms == 3) return launch_one<0, 3>(d_inst, d_tiles, n_tiles, d_maxbits, cfg, d_status, s);
    if (cfg.elem == 1 && cfg.terms == 3) return launch_one<1, 3>(d_inst, d_tiles, n_tiles, d_maxbits, cfg, d_status, s);
    if (cfg.elem == 0 && cfg.terms == 1) return launch_one<0, 1>(d_inst, d_tiles, n_tiles, d_maxbits, cfg, d_status, s);
    if (cfg.elem == 1 && cfg.terms == 1) return launch_one<1, 1>(d_inst, d_tiles, n_tiles, d_maxbits, cfg, d_status, s);
    return cudaErrorNotSupported;
}

}  // namespace laph
