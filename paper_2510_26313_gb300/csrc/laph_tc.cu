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
// K stages (chunk_stages_b for tiles without meson rows, whose incoherent
// sums tolerate a longer interval) into a second tensor-memory region of
// FP32 running sums kept by CUDA cores with round-to-nearest.  A tile covers
// one block of sites (at most sc_stages K stages); at its end the running
// sums are stored as FP32 partials, and reduce_kernel adds the partials of
// all site blocks of an output in FP64, in block order, scales them back and
// writes the complex128 (or complex64) output.  At chunk boundaries the MMAs of the two column halves
// of the accumulator are issued and committed separately, so that the drain
// of one half overlaps the MMAs of the other.
//
// Tile: 128 rows x 104 complex columns by default (UMMA M = 128, N = 208, the
// widest that fits; 96, 80 and 64 columns, and 64 rows x 208, 192, 176 or
// 128 columns in the row-doubled layout, are the other shapes).  A K stage
// is one site block: TC_BS = 8 sites = 24 complex = 48 real K entries, three
// MMA k-steps of 16.
// Tensor memory (512 columns): ACC [0,N) | SUM [N,2N) | two A slots of 48
// from column 416 (hi in 24 columns, lo in the next 24).
//
// The B operand does not depend on the row tile, so psi_kernel builds it
// once per (timeslice, column tile): a memory-bound pass that writes every
// stage as the exact image of a shared-memory B stage (hi and lo, K-major,
// 32-byte swizzle: one swizzle atom column per k-step).  The contraction's
// stage ring holds, per stage, that image and the block slots of the tile's
// row vectors (from the site-blocked, pre-scaled copy of phi); one loader
// warp fills a stage with two bulk copies completing on one mbarrier, and
// the MMA's commit frees it.
//
// Warp roles (persistent CTAs; the loader claims tiles from a global counter
// and hands them to the other roles through a small ring):
//   0-15  A producers in two groups of eight; group g forms the stages whose
//         global index has parity g, in A slot g, so that two stages are
//         formed at once.  Within a group, two warps per TMEM lane quadrant:
//         warp half h forms the 12 K entries of sites 4h..4h+3 of its row
//         (diquark or conj(phi)), splits them and tcgen05.st's them;
//   16-23 epilogue, two warps per TMEM lane quadrant taking alternate blocks
//         of 16 columns (row-doubled layout: 16-19, one per quadrant): drains
//         ACC into SUM, one column half at a time, writes the FP32 partials
//         at tile end;
//   then  the loader: claims the next tile, then the stage ring's bulk
//         copies; and TMEM allocation and single-thread MMA issue.
// 26 warps (832 threads, at most 72 registers a thread so that seven warps
// fit one scheduler's register file); the row-doubled layout keeps 22 warps
// (one epilogue warp per quadrant) at 80 registers, which measured faster
// there.
// Every wait on an mbarrier is bounded; on expiry the CTA records
// STATUS_TIMEOUT, raises a shared abort flag and all roles return.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "laph_internal.cuh"

namespace laph {
namespace {

constexpr int N_AGROUP = 8;                           // A producer warps per group (one stage)
constexpr int N_AWARPS = 2 * N_AGROUP;
// Warp counts of the two layouts: the epilogue warps (two per lane quadrant
// halve the drain time) and the loader and MMA warps after them.
template <bool RD>
struct Roles {
    static constexpr int EPI_WARPS = RD ? 4 : 8;
    static constexpr int WARP_LOAD = N_AWARPS + EPI_WARPS;
    static constexpr int WARP_MMA = WARP_LOAD + 1;
    static constexpr int NTHREADS = (WARP_MMA + 1) * 32;
    static constexpr int N_TILE_READERS = N_AWARPS + EPI_WARPS + 1;   // A producers, epilogue, MMA
};
constexpr int KSTAGE = TC_KSTAGE;                     // complex K entries per stage (one site block)
constexpr int KSTEPS = 2 * KSTAGE / 16;               // MMA k-steps per stage
constexpr int SLOT_BYTES = TC_SLOT * 8;               // 208 B = 52 words: LDS.128 of 8 consecutive slots hit distinct banks
constexpr int HALF_BYTES = (TC_BS / 2) * 3 * 8;       // 4 sites x 3 colours: one A warp's share of a slot
constexpr int MAX_NS = 6;
constexpr int TRING = 4;                              // tile ring entries
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t ACC_COL = 0;
constexpr uint32_t A_COL = 416;
constexpr uint32_t A_SLOT_COLS = 48;
constexpr uint32_t A_LO = KSTAGE;                     // lo columns follow the 24 hi columns
constexpr long long WAIT_LIMIT = 4000000000LL;        // cycles (about 2 s at the top clock)

static_assert(TC_TR == 128, "layout assumes 128-row tiles (UMMA M = 128, one tensor-memory lane per row)");
static_assert(TC_BS == 8 && KSTAGE == 24 && KSTEPS == 3, "a stage is one 8-site block");
static_assert(A_LO + KSTAGE <= A_SLOT_COLS && A_COL + 2 * A_SLOT_COLS == TMEM_COLS, "tensor memory budget");

// Sizes that follow from the tile width NC (complex columns) and the layout
// of the complex product.  RD false: every complex column is two real B rows
// (re-row, im-row), UMMA N = 2 NC, and a tile has 128 complex rows; RD true:
// every complex row r is two real A rows (tensor-memory lanes r and 64 + r), UMMA
// N = NC, and a tile has 64 complex rows.  Tensor memory: the accumulator in
// columns [0, B_ROWS), the FP32 running sums in [B_ROWS, 2 B_ROWS), the two
// A slots from column 416.
template <int NC, bool RD>
struct Shape {
    static constexpr int B_ROWS = RD ? NC : 2 * NC;        // real B rows per tile (UMMA N)
    static constexpr int ATOM_COL_BYTES = (B_ROWS / 8) * 256;   // one k-step of hi (or lo): atoms of 8 rows x 32 B
    static constexpr int B_BYTES = KSTEPS * ATOM_COL_BYTES;     // hi (or lo) of one stage
    static constexpr int BIMG_BYTES = 2 * B_BYTES;              // hi + lo
    static constexpr uint32_t SUM_COL = B_ROWS;
    static_assert(B_ROWS % 16 == 0 && B_ROWS <= 208 && 2 * B_ROWS <= (int)A_COL,
                  "tile width within the tensor-memory budget");
    static_assert(BIMG_BYTES == tc_stage_bytes(NC, RD), "stage image size");
};

// Accumulator columns of a tile (UMMA N): its valid columns rounded up, less
// the leading columns no row needs (RD: multiples of 16 complex columns, one
// real B row each; otherwise multiples of 8, two real B rows each).
template <bool RD>
__device__ __forceinline__ int acc_cols(int ncols, int cskip)
{
    return RD ? ((ncols + 15) & ~15) - cskip : 2 * ((ncols + 7) & ~7) - 2 * cskip;
}

struct Shared {
    // full: data of stage k landed, barrier k mod 2 NS (every barrier serves
    // one A-producer group only, even when NS is odd); empty: stage k's MMAs
    // done, barrier k mod NS (the stage buffer)
    uint64_t full[2 * MAX_NS], empty[MAX_NS];
    uint64_t tfull[TRING], tempty[TRING];
    int tile_ring[TRING];
    uint64_t a_full[2];
    uint64_t acc_full[2], acc_empty[2];   // per column half of the accumulator
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

// Tests the phase with the given parity for completion; the warp may be
// suspended for a system-dependent time while it is incomplete.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
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

__device__ __forceinline__ void tmem_st4(uint32_t taddr, uint32_t v0, uint32_t v1, uint32_t v2, uint32_t v3)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(v0), "r"(v1),
                 "r"(v2), "r"(v3)
                 : "memory");
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

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 32-byte swizzle, 8-row groups
// 256 bytes apart (SBO), version 1.  One swizzle atom (8 rows x 32 bytes)
// spans the 16 K entries of one MMA k-step.
__device__ __forceinline__ uint64_t desc_sw32(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(16u >> 4) << 16;
    d |= (uint64_t)(256u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)6 << 61;
    return d;
}

// Instruction descriptor, kind::f16: FP32 D, FP16 (0) or BF16 (1) A and B,
// both K-major, M = 128, N = n_real.
__device__ __forceinline__ uint32_t idesc_f16(int n_real, int bf16)
{
    return (1u << 4) | ((uint32_t)bf16 << 7) | ((uint32_t)bf16 << 10) | ((uint32_t)(n_real >> 3) << 17) |
           ((uint32_t)(128 >> 4) << 24);
}

// Byte offset of 16-byte chunk j (0, 1) of real row n inside one k-step's
// atom column of a stage image (32-byte swizzle: chunk bit ^= row bit 2).
__device__ __forceinline__ uint32_t sw32(int n, int j)
{
    return (uint32_t)((n >> 3) * 256 + (n & 7) * 32 + ((j ^ ((n >> 2) & 1)) << 4));
}

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

// ------------------------------------------------------------ waits

struct Ctx {
    Shared *S;
    int *status;
    int lane;
};

// Slow path of a warp-wide bounded wait.  Between the try_waits (each may
// suspend the warp for a while) the abort flag and the time limit are
// checked.
__device__ __noinline__ bool warp_wait_slow(Shared *S, int *status, int lane, uint64_t *bar, uint32_t parity)
{
    const long long t0 = clock64();
    while (true) {
        if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;
        const int ab = *(volatile int *)&S->abort;
        if (__any_sync(0xffffffffu, ab != 0)) return false;
        int expired = (clock64() - t0) > WAIT_LIMIT;
        expired = __shfl_sync(0xffffffffu, expired, 0);
        if (expired) {
            if (lane == 0) {
                *(volatile int *)&S->abort = 1;
                atomicOr(status, STATUS_TIMEOUT);
            }
            return false;
        }
    }
}

// Bounded wait that ignores the abort flag: used at exit to let the bulk
// copies a warp issued land before the CTA's shared memory is released.
__device__ __noinline__ void drain_wait(Shared *S, int *status, int lane, uint64_t *bar, uint32_t parity)
{
    const long long t0 = clock64();
    while (!__all_sync(0xffffffffu, mbar_try_wait(bar, parity))) {
        if (clock64() - t0 > WAIT_LIMIT) {
            if (lane == 0) {
                *(volatile int *)&S->abort = 1;
                atomicOr(status, STATUS_TIMEOUT);
            }
            return;
        }
    }
}

// Warp-wide bounded wait (every lane calls it; the result is warp-uniform).
__device__ __forceinline__ bool warp_wait(const Ctx c, uint64_t *bar, uint32_t parity)
{
    if (__all_sync(0xffffffffu, mbar_try_wait(bar, parity))) return true;
    return warp_wait_slow(c.S, c.status, c.lane, bar, parity);
}

// Ring position: slot index and the parity of its current phase.
struct Ring {
    int slot;
    uint32_t phase;
    __device__ __forceinline__ void next(int n)
    {
        if (++slot == n) {
            slot = 0;
            phase ^= 1u;
        }
    }
};

// Next tile of this CTA from the tile ring (-1: no more tiles).  Every
// reader warp takes every entry in order and frees it at once.
__device__ __forceinline__ int next_tile(const Ctx c, Ring &rt, bool &ok)
{
    if (!warp_wait(c, &c.S->tfull[rt.slot], rt.phase)) {
        ok = false;
        return -1;
    }
    const int t = *(volatile int *)&c.S->tile_ring[rt.slot];
    __syncwarp();
    if (c.lane == 0) mbar_arrive(&c.S->tempty[rt.slot]);
    rt.next(TRING);
    return t;
}

// ------------------------------------------------------------ A producer

// The 12 K entries of sites 4h..4h+3 of one row, from the block slots of
// phi_i (pu) and phi_j (pv), split into hi and lo words.  kind: 2 diquark,
// 1 meson (conj(phi_i)), 0 no row (zeros).  FORM: how an entry x of the
// complex operand becomes a pair of real K entries: 0 (re, im), the
// column-doubled layout; in the row-doubled layout 1 (re, -im) for the re-row
// and 2 (im, re) for the im-row of a complex row, so that with B rows
// (Psi_re, Psi_im) the re-row gives the real part of the product and the
// im-row its imaginary part.
template <int ELEM, int FORM>
__device__ __forceinline__ void a_quarter(int kind, const uint8_t *pu, const uint8_t *pv, uint32_t (&hi)[12],
                                          uint32_t (&lo)[12])
{
#pragma unroll
    for (int m = 0; m < 2; m++) {
        // two sites = 6 entries = three 16-byte loads per vector
        float2 u[6], v[6];
#pragma unroll
        for (int h = 0; h < 3; h++) {
            const float4 a = reinterpret_cast<const float4 *>(pu)[3 * m + h];
            const float4 b = reinterpret_cast<const float4 *>(pv)[3 * m + h];
            u[2 * h] = make_float2(a.x, a.y);
            u[2 * h + 1] = make_float2(a.z, a.w);
            v[2 * h] = make_float2(b.x, b.y);
            v[2 * h + 1] = make_float2(b.z, b.w);
        }
#pragma unroll
        for (int e = 0; e < 6; e++) {
            float2 d;
            if (kind == 2)
                d = cross8(u + 3 * (e / 3), v + 3 * (e / 3), e % 3);
            else if (kind == 1)
                d = make_float2(u[e].x, -u[e].y);
            else
                d = make_float2(0.f, 0.f);
            if (FORM == 1) d = make_float2(d.x, -d.y);
            if (FORM == 2) d = make_float2(d.y, d.x);
            split2<ELEM>(d.x, d.y, hi[6 * m + e], lo[6 * m + e]);
        }
    }
}

// hi words to columns ta..ta+11, lo words to ta + A_LO ..
__device__ __forceinline__ void a_store(uint32_t ta, const uint32_t (&hi)[12], const uint32_t (&lo)[12])
{
#pragma unroll
    for (int q = 0; q < 3; q++) {
        tmem_st4(ta + 4 * q, hi[4 * q], hi[4 * q + 1], hi[4 * q + 2], hi[4 * q + 3]);
        tmem_st4(ta + A_LO + 4 * q, lo[4 * q], lo[4 * q + 1], lo[4 * q + 2], lo[4 * q + 3]);
    }
}

// ------------------------------------------------------------ the kernel

struct KParams {
    const InstDev *insts;
    const TileDev *tiles;
    const unsigned *maxbits;
    const uint8_t *psi;   // B stage images of the chunk
    float2 *part;         // FP32 partial sums of the chunk's site blocks
    unsigned *counter;    // tile counter of this launch (zero at launch)
    int *status;
    int n_tiles;
    int chunk_stages;     // drain interval in K stages
    int chunk_stages_b;   // the same for tiles without meson rows
    int stage_bytes;      // one stage buffer: B image, then the row vectors' block slots
    int ns;               // stage buffers
    int debug_stall;
};

template <int ELEM, int TERMS, int NC, bool RD>
__global__ void __launch_bounds__(Roles<RD>::NTHREADS, 1) tc_kernel(const KParams kp)
{
    using SH = Shape<NC, RD>;
    using R = Roles<RD>;
    constexpr int WARP_LOAD = R::WARP_LOAD, WARP_MMA = R::WARP_MMA, N_TILE_READERS = R::N_TILE_READERS;
    constexpr int BIMG_BYTES = SH::BIMG_BYTES, B_BYTES = SH::B_BYTES, ATOM_COL_BYTES = SH::ATOM_COL_BYTES;
    constexpr uint32_t SUM_COL = SH::SUM_COL;
    extern __shared__ uint8_t smem_raw[];
    // align to 1024 bytes by offsetting the __shared__ array itself, so that
    // the compiler keeps every derived pointer in the shared address space
    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const int NS = kp.ns;
    Shared *S = reinterpret_cast<Shared *>(smem + NS * kp.stage_bytes);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Ctx c{S, kp.status, lane};

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; s++) {
            mbar_init(&S->full[s], 1);
            mbar_init(&S->full[NS + s], 1);
            mbar_init(&S->empty[s], 1);
        }
        for (int s = 0; s < TRING; s++) {
            mbar_init(&S->tfull[s], 1);
            mbar_init(&S->tempty[s], N_TILE_READERS);
        }
        for (int s = 0; s < 2; s++) {
            mbar_init(&S->a_full[s], N_AGROUP);
        }
        for (int h = 0; h < 2; h++) {
            mbar_init(&S->acc_full[h], 1);
            mbar_init(&S->acc_empty[h], R::EPI_WARPS);
        }
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
        Ring rs{0, 0}, rf{0, 0}, rt{0, 0};   // stage buffer, data barrier, tile ring
        uint32_t n_issued = 0;   // stages whose copies were issued
        bool ok = true;
        while (ok) {
            if (!warp_wait(c, &S->tempty[rt.slot], rt.phase ^ 1u)) break;
            int tile = 0;
            if (lane == 0) {
                tile = (int)atomicAdd(kp.counter, 1u);
                if (tile >= kp.n_tiles) tile = -1;
                *(volatile int *)&S->tile_ring[rt.slot] = tile;
                mbar_arrive(&S->tfull[rt.slot]);
            }
            tile = __shfl_sync(0xffffffffu, tile, 0);
            rt.next(TRING);
            if (tile < 0) break;
            const TileDev td = kp.tiles[tile];
            const InstDev &I = kp.insts[td.inst];
            const int nst = td.nst;
            // row vectors: [v_lo, v_lo + nv) of phi_u, then (triplets) [w_lo, w_lo + nw) of phi_v,
            // from site block s0 of the tile's site range on
            const uint32_t bytesA = td.nv * SLOT_BYTES, bytesW = td.nw * SLOT_BYTES;
            const uint8_t *bsrc = kp.psi + td.psi_off + (long long)td.s0 * BIMG_BYTES;
            const long long blk0 = ((long long)td.t * I.nblk + td.s0) * I.N;
            const float2 *asrc = I.phi_blk + (blk0 + td.v_lo) * TC_SLOT;
            const float2 *wsrc = I.blk_v + (blk0 + td.w_lo) * TC_SLOT;
            const long long astep = (long long)I.N * TC_SLOT;
            for (int st = 0; st < nst; st++) {
                if (!warp_wait(c, &S->empty[rs.slot], rs.phase ^ 1u)) {
                    ok = false;
                    break;
                }
                if (lane == 0) {
                    uint8_t *buf = smem + rs.slot * kp.stage_bytes;
                    uint64_t *fb = &S->full[rf.slot];
                    mbar_arrive_expect_tx(fb, BIMG_BYTES + bytesA + bytesW);
                    bulk_g2s(buf, bsrc + (long long)st * BIMG_BYTES, BIMG_BYTES, fb);
                    bulk_g2s(buf + BIMG_BYTES, asrc + st * astep, bytesA, fb);
                    if (bytesW) bulk_g2s(buf + BIMG_BYTES + bytesA, wsrc + st * astep, bytesW, fb);
                }
                __syncwarp();
                rs.next(NS);
                rf.next(2 * NS);
                n_issued++;
            }
        }
        // the copies of the last NS issued stages may still be in flight (after
        // an abort nobody consumed them): wait until they have landed
        for (uint32_t k = n_issued > (uint32_t)NS ? n_issued - NS : 0; k < n_issued; k++)
            drain_wait(S, kp.status, lane, &S->full[k % (2 * NS)], (k / (2 * NS)) & 1u);
    } else if (warp < N_AWARPS) {
        // ---------------------------------------------------------- A producers
        const int quad = warp & 3, half = (warp >> 2) & 1, grp = warp >> 3;
        // the lane's (complex) row of the tile; row-doubled layout: lane quadrants 0, 1 hold the re-rows of the
        // tile's 64 complex rows, quadrants 2, 3 their im-rows
        const int r = RD ? 32 * (quad & 1) + lane : quad * 32 + lane;
        const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
        const uint32_t ta0 = tmem + lane_base + A_COL + (uint32_t)grp * A_SLOT_COLS + 12u * half;
        uint32_t G = 0;   // global index of the tile's first stage
        bool stalled = false, ok = true;
        Ring rt{0, 0};
        while (ok) {
            const int tile = next_tile(c, rt, ok);
            if (tile < 0) break;
            const TileDev td = kp.tiles[tile];
            const InstDev &I = kp.insts[td.inst];
            const int nst = td.nst;
            const int gr = td.row0 + r;
            int kind = 0, vi = 0, vj = 0;
            const bool trip = I.kind == INST_TRIPLETS;
            if (gr < I.rows) {
                if (gr < I.mes_rows) {
                    kind = 1;
                    vi = gr;
                } else {
                    kind = 2;
                    const int q = gr - I.mes_rows;
                    if (trip) {
                        vi = q / I.N;
                        vj = q - vi * I.N;
                    } else {
                        pair_of(q, vi, vj);
                    }
                }
            }
            // staged slots: phi_u vector vi, and phi_v vector vj (the same staged
            // vectors unless triplets, whose phi_v slots follow the nv phi_u slots)
            const int si = kind ? vi - td.v_lo : 0;
            const int sj = kind == 2 ? (trip ? td.nv + vj - td.w_lo : vj - td.v_lo) : 0;
            const int off_u = BIMG_BYTES + si * SLOT_BYTES + half * HALF_BYTES;
            const int off_v = BIMG_BYTES + sj * SLOT_BYTES + half * HALF_BYTES;
            // this group's stages: global index Gs = G + st with parity grp
            int st = (grp - (int)(G & 1u)) & 1;
            const uint32_t Gs = G + st;
            int s = (int)(Gs % (uint32_t)NS);        // stage buffer
            int sf = (int)(Gs % (uint32_t)(2 * NS)); // its data barrier: used by this group only,
            uint32_t ph = (Gs / (uint32_t)(2 * NS)) & 1u;  // one phase per use, in order
            // A slot grp is free once stage Gs - 2, its previous user, has
            // completed: the stage's commit to empty[(Gs - 2) mod NS].  Before
            // the first use the parity wait passes on the fresh barrier.
            const uint32_t Gp = Gs + (uint32_t)NS - 2u;
            int s2 = (int)(Gp % (uint32_t)NS);
            uint32_t ph2 = ((Gp / (uint32_t)NS) & 1u) ^ 1u;
            for (; st < nst; st += 2) {
                // the entries are formed as soon as the stage has landed; only
                // the stores into the A slot wait for the MMAs reading it
                if (!warp_wait(c, &S->full[sf], ph)) {
                    ok = false;
                    break;
                }
                const uint8_t *buf = smem + s * kp.stage_bytes;
                uint32_t hi[12], lo[12];
                if (!RD)
                    a_quarter<ELEM, 0>(kind, buf + off_u, buf + off_v, hi, lo);
                else if (quad < 2)
                    a_quarter<ELEM, 1>(kind, buf + off_u, buf + off_v, hi, lo);
                else
                    a_quarter<ELEM, 2>(kind, buf + off_u, buf + off_v, hi, lo);
                if (!warp_wait(c, &S->empty[s2], ph2)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                a_store(ta0, hi, lo);
                tmem_wait_st();
                tc_fence_before();
                __syncwarp();
                const bool skip = kp.debug_stall && !stalled && blockIdx.x == 0 && warp == 0;
                if (skip) stalled = true;
                if (lane == 0 && !skip) mbar_arrive(&S->a_full[grp]);
                s += 2;
                if (s >= NS) s -= NS;
                sf += 2;
                if (sf >= 2 * NS) {
                    sf -= 2 * NS;
                    ph ^= 1u;
                }
                s2 += 2;
                if (s2 >= NS) {
                    s2 -= NS;
                    ph2 ^= 1u;
                }
            }
            G += (uint32_t)nst;
        }
    } else if (warp < WARP_LOAD) {
        // ---------------------------------------------------------- epilogue
        const int quad = warp & 3;
        constexpr int N_EH = R::EPI_WARPS / 4;            // epilogue warps per lane quadrant
        const int eh = (warp - N_AWARPS) >> 2;            // this warp's share: 16-column blocks b with b % N_EH == eh
        const int r = RD ? 32 * (quad & 1) + lane : quad * 32 + lane;   // the lane's (complex) row of the tile
        const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
        uint32_t gc = 0, gc1 = 0;   // drains done of the low / high column half
        bool ok = true;
        Ring rt{0, 0};
        while (ok) {
            const int tile = next_tile(c, rt, ok);
            if (tile < 0) break;
            const TileDev td = kp.tiles[tile];
            const InstDev &I = kp.insts[td.inst];
            const int ncols = td.ncols, cskip = td.cskip;
            const int n_real = acc_cols<RD>(ncols, cskip);   // accumulator columns: tile columns cskip..
            const int gr = td.row0 + r;
            const bool rvalid = gr < I.rows;
            const bool meson = gr < I.mes_rows;
            const bool trip = I.kind == INST_TRIPLETS;
            int pi_ = 0, pj = 0;
            long long q = 0;
            if (rvalid && !meson) {
                q = gr - I.mes_rows;
                if (trip) {
                    pi_ = (int)(q / I.N);
                    pj = (int)(q - (long long)pi_ * I.N);
                } else {
                    pair_of(q, pi_, pj);
                }
            }
            const int cs = td.row0 >= I.mes_rows ? kp.chunk_stages_b : kp.chunk_stages;   // drain interval
            const int n_ch = (td.nst + cs - 1) / cs;
            const int n_lo = n_real >= 32 ? ((n_real / 2 + 15) & ~15) : n_real;
            for (int ch = 0; ch < n_ch && ok; ch++) {
                for (int h = 0; h < 2; h++) {
                    const int c0 = h ? n_lo : 0, c1 = h ? n_real : n_lo;
                    if (c1 <= c0) continue;
                    uint32_t &g = h ? gc1 : gc;
                    if (!warp_wait(c, &S->acc_full[h], g & 1u)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    for (int b = c0 / 16; b * 16 < c1; b++) {
                        if (N_EH > 1 && b % N_EH != eh) continue;
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
                    if (lane == 0) mbar_arrive(&S->acc_empty[h]);
                    g++;
                }
            }
            if (!ok) break;
            // tile done: the FP32 sums of its site block go to the partial
            // buffer in the output order of one timeslice (B entries, then M
            // entries), still scaled; the FP64 reduction over site blocks
            // scales them back
            const int P = I.P, N = I.N;
            const long long n_trip = I.n_trip;
            float2 *part = kp.part + td.part_off;
            for (int b = 0; b * 16 < n_real; b++) {
                if (N_EH > 1 && b % N_EH != eh) continue;
                uint32_t v[16];
                tmem_ld16(tmem + lane_base + SUM_COL + 16u * b, v);
                tmem_wait_ld();
                if (RD) {
                    // lane quadrants 0, 1 hold the real parts of the complex
                    // rows, quadrants 2, 3 the imaginary parts: each writes its half
#pragma unroll
                    for (int u = 0; u < 16; u++) {
                        const int cc = cskip + 16 * b + u;
                        if (!rvalid || cc >= ncols) continue;
                        const int col = td.col0 + cc;
                        const int k = col / P, p = col - k * P;
                        long long e;
                        if (meson) {
                            e = I.n_outB + ((long long)p * N + gr) * I.Nc + k;
                        } else if (trip) {
                            e = (((long long)p * N + pi_) * N + pj) * N + k;
                        } else {
                            if (k <= pj) continue;
                            e = (long long)p * n_trip + binom3(k) + q;
                        }
                        reinterpret_cast<float *>(part + e)[quad >> 1] = __uint_as_float(v[u]);
                    }
                    continue;
                }
#pragma unroll 1
                for (int u = 0; u < 8; u++) {
                    const int cc = cskip + 8 * b + u;
                    if (!rvalid || cc >= ncols) continue;
                    const int col = td.col0 + cc;
                    const int k = col / P, p = col - k * P;
                    long long e;
                    if (meson) {
                        e = I.n_outB + ((long long)p * N + gr) * I.Nc + k;   // [p][i][k], k < Nc
                    } else if (trip) {
                        e = (((long long)p * N + pi_) * N + pj) * N + k;    // dense [p][i][j][k]
                    } else {
                        if (k <= pj) continue;
                        e = (long long)p * n_trip + binom3(k) + q;
                    }
                    part[e] = make_float2(__uint_as_float(v[2 * u]), __uint_as_float(v[2 * u + 1]));
                }
            }
        }
    } else {
        // ---------------------------------------------------------- MMA issue
        Ring rs{0, 0}, ra{0, 0};
        uint32_t gc = 0, gc1 = 0;   // chunks of the low / high column half
        bool issued = false, ok = true;
        Ring rt{0, 0};
        while (ok) {
            const int tile = next_tile(c, rt, ok);
            if (tile < 0) break;
            const TileDev td = kp.tiles[tile];
            const int nst = td.nst;
            const int chunk = td.row0 >= kp.insts[td.inst].mes_rows ? kp.chunk_stages_b : kp.chunk_stages;
            // the first cskip columns (2 cskip real B rows, or cskip in the
            // row-doubled layout; 32 bytes per B row in every atom column) are
            // not needed by any row of the tile
            const int n_real = acc_cols<RD>(td.ncols, td.cskip);
            const uint32_t idesc = idesc_f16(n_real, ELEM);
            const uint64_t bskip = (uint64_t)(td.cskip * (RD ? 32 : 64)) >> 4;
            // column halves [0, n_lo) and [n_lo, n_real) of the accumulator
            const int n_lo = n_real >= 32 ? ((n_real / 2 + 15) & ~15) : n_real;
            const int nh = n_real > n_lo ? 2 : 1;
            const uint32_t idesc_h[2] = {idesc_f16(n_lo, ELEM), nh == 2 ? idesc_f16(n_real - n_lo, ELEM) : 0u};
            int cs = 0;   // stage within the current accumulation chunk
            for (int st = 0; st < nst; st++) {
                const bool chunk_start = cs == 0;
                const bool chunk_end = cs + 1 == chunk || st + 1 == nst;
                // Every producer warp of the stage waited for the stage's data
                // (its full barrier) before its release-arrive on a_full, so the
                // acquire of a_full also orders the MMAs after the bulk copies;
                // the MMA warp waits on one barrier per stage.
                if (!warp_wait(c, &S->a_full[ra.slot], ra.phase)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t a_hi = tmem + A_COL + (uint32_t)ra.slot * A_SLOT_COLS, a_lo = a_hi + A_LO;
                // descriptor start addresses advance one atom column (in units of 16 bytes) per k-step
                const uint64_t dhi = desc_sw32(smem_u32(smem + rs.slot * kp.stage_bytes)) + bskip;
                const uint64_t dlo = dhi + (uint64_t)(B_BYTES >> 4);
                if (!chunk_start && !chunk_end) {
                    if (lane == 0) {
#pragma unroll
                        for (int ks = 0; ks < KSTEPS; ks++) {
                            const uint64_t koff = (uint64_t)ks * (ATOM_COL_BYTES >> 4);
                            mma_ts(tmem + ACC_COL, a_hi + 8 * ks, dhi + koff, idesc, 1u);
                            if (TERMS == 3) {
                                mma_ts(tmem + ACC_COL, a_hi + 8 * ks, dlo + koff, idesc, 1u);
                                mma_ts(tmem + ACC_COL, a_lo + 8 * ks, dhi + koff, idesc, 1u);
                            }
                        }
                    }
                } else {
                    for (int h = 0; h < nh && ok; h++) {
                        uint32_t &g = h ? gc1 : gc;
                        if (chunk_start) {
                            if (!warp_wait(c, &S->acc_empty[h], (g & 1u) ^ 1u)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                        }
                        if (lane == 0) {
                            // half h: accumulator columns and B rows from h * n_lo (32 bytes per row per atom column)
                            const uint32_t d = tmem + ACC_COL + (uint32_t)(h * n_lo);
                            const uint64_t hoff = (uint64_t)(h * n_lo * 32) >> 4;
#pragma unroll
                            for (int ks = 0; ks < KSTEPS; ks++) {
                                const uint32_t acc = (chunk_start && ks == 0) ? 0u : 1u;
                                const uint64_t koff = (uint64_t)ks * (ATOM_COL_BYTES >> 4) + hoff;
                                mma_ts(d, a_hi + 8 * ks, dhi + koff, idesc_h[h], acc);
                                if (TERMS == 3) {
                                    mma_ts(d, a_hi + 8 * ks, dlo + koff, idesc_h[h], 1u);
                                    mma_ts(d, a_lo + 8 * ks, dhi + koff, idesc_h[h], 1u);
                                }
                            }
                            if (chunk_end) mma_commit(&S->acc_full[h]);
                        }
                        __syncwarp();
                        if (chunk_end) g++;
                    }
                    if (!ok) break;
                }
                if (lane == 0) {
                    // one commit frees the stage buffer (loader) and the A slot (producers)
                    mma_commit(&S->empty[rs.slot]);
                    issued = true;
                }
                __syncwarp();
                cs = chunk_end ? 0 : cs + 1;
                rs.next(NS);
                ra.next(2);
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

// ------------------------------------------------------------ B stage images

// Job = (unit, column tile ct, group of TC_PSI_GROUP consecutive stages); the
// unit is the last one whose job0 <= job.  Thread (cu = tid / 2, j = tid % 2)
// takes tile column cu (complex column col0 + cu = k * P + p) and, for every
// stage st of the group and k-step ks, the four K entries
// kap = 24 st + 8 ks + 4 j + v (v < 4, site x = kap / 3, colour kap % 3):
// Psi = ph_p(x) * (2^s phi_k(x, c)) -- zero past K or past the last column --
// is split into hi/lo and stored as 16-byte chunk j of the re-row (re, -im)
// at real row 2 cu and of the im-row (im, re) at row 2 cu + 1 of the stage
// image, in the K-major 32-byte-swizzled layout the contraction's
// descriptors expect.  Every store instruction of a warp writes sixteen
// whole 32-byte rows.
template <int ELEM, int NC, bool RD>
__global__ void __launch_bounds__(2 * NC) psi_kernel(const InstDev *__restrict__ insts, const PsiUnit *__restrict__ units,
                                                     int n_units, long long n_jobs, const unsigned *__restrict__ maxbits,
                                                     uint8_t *__restrict__ psi)
{
    using SH = Shape<NC, RD>;
    constexpr int BIMG_BYTES = SH::BIMG_BYTES, B_BYTES = SH::B_BYTES, ATOM_COL_BYTES = SH::ATOM_COL_BYTES;
    const int cu = threadIdx.x >> 1, j = threadIdx.x & 1;
    for (long long job = blockIdx.x; job < n_jobs; job += gridDim.x) {
        int lo = 0, hi = n_units - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (units[mid].job0 <= job)
                lo = mid;
            else
                hi = mid - 1;
        }
        const PsiUnit un = units[lo];
        const InstDev &I = insts[un.inst];
        const int n_st = I.n_st;
        const int n_grp = (n_st + TC_PSI_GROUP - 1) / TC_PSI_GROUP;
        const int jl = (int)(job - un.job0);
        const int ct = jl / n_grp;
        const int st0 = (jl - ct * n_grp) * TC_PSI_GROUP;
        const int st1 = min(st0 + TC_PSI_GROUP, n_st);
        const int col0 = ct * NC;
        const bool valid = cu < min(NC, I.cols - col0);
        const int V = (int)I.V;
        const float sc = pow2f(scale_exp(maxbits[I.ts_base + un.t]));
        int k = 0, p = 0;
        if (valid) {
            k = (col0 + cu) / I.P;
            p = col0 + cu - k * I.P;
        }
        const float2 *ph = I.phase + (long long)p * I.Vs;
        const float2 *phk = I.phi + ((long long)un.t * I.Nc + k) * V * 3;
        uint8_t *img = psi + un.psi_off + ((long long)ct * n_st + st0) * BIMG_BYTES;
        // real B rows of the column: re-row 2 cu and im-row 2 cu + 1, or (row-doubled layout) row cu
        const int n0 = RD ? cu : 2 * cu, n1 = n0 + 1;
        const uint32_t o0 = sw32(n0, j), o1 = sw32(n1, j);
        for (int st = st0; st < st1; st++, img += BIMG_BYTES) {
#pragma unroll
            for (int ks = 0; ks < KSTEPS; ks++) {
                // entries e0 .. e0+3 of the stage: sites 8 st + (e0 + v) / 3
                const int e0 = 8 * ks + 4 * j;
                const int xs = 8 * st + e0 / 3, c0 = e0 % 3;
                float2 f[4], w[2];
#pragma unroll
                for (int v = 0; v < 4; v++) {
                    const int x = xs + (c0 + v) / 3;
                    f[v] = (valid && x < V) ? __ldg(phk + 3 * x + (c0 + v) % 3) : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int q = 0; q < 2; q++) w[q] = (valid && xs + q < V) ? __ldg(ph + xs + q) : make_float2(0.f, 0.f);
                uint32_t rh[4], rl[4], ih[4], il[4];
#pragma unroll
                for (int v = 0; v < 4; v++) {
                    const float2 z = cmulf(w[(c0 + v) / 3], make_float2(f[v].x * sc, f[v].y * sc));
                    uint32_t h, l;
                    split2<ELEM>(z.x, z.y, h, l);
                    if (RD) {
                        rh[v] = h;                          // (re, im)
                        rl[v] = l;
                    } else {
                        rh[v] = h ^ 0x80000000u;            // (re, -im)
                        rl[v] = l ^ 0x80000000u;
                        ih[v] = __byte_perm(h, 0, 0x1032);  // (im, re)
                        il[v] = __byte_perm(l, 0, 0x1032);
                    }
                }
                uint8_t *out = img + ks * ATOM_COL_BYTES;
                if (RD) {
                    *reinterpret_cast<uint4 *>(out + o0) = make_uint4(rh[0], rh[1], rh[2], rh[3]);
                    *reinterpret_cast<uint4 *>(out + B_BYTES + o0) = make_uint4(rl[0], rl[1], rl[2], rl[3]);
                    continue;
                }
                *reinterpret_cast<uint4 *>(out + o0) = make_uint4(rh[0], rh[1], rh[2], rh[3]);
                *reinterpret_cast<uint4 *>(out + o1) = make_uint4(ih[0], ih[1], ih[2], ih[3]);
                *reinterpret_cast<uint4 *>(out + B_BYTES + o0) = make_uint4(rl[0], rl[1], rl[2], rl[3]);
                *reinterpret_cast<uint4 *>(out + B_BYTES + o1) = make_uint4(il[0], il[1], il[2], il[3]);
            }
        }
    }
}

// ------------------------------------------------------------ FP64 site reduction

// Exact FP32 -> FP64 widening done on the integer units (GB300 runs FP64
// instructions at a small fraction of the FP32 rate, so the reduction keeps
// its FP64 instructions to the additions): a normal float's sign, exponent
// (rebiased by 1023 - 127) and mantissa are placed in the double's fields;
// zeros, subnormals and non-finite values take the hardware conversion.
__device__ __forceinline__ double widen(float f)
{
    const uint32_t u = __float_as_uint(f);
    const uint32_t ex = (u >> 23) & 0xffu;
    if (ex == 0u || ex == 0xffu) return (double)f;
    const unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                                 ((unsigned long long)(ex + 896u) << 52) | ((unsigned long long)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)b);
}

// v * 2^k for the exact power-of-two rescale, by adding k to the exponent
// field when the result stays a normal number (else one multiplication).
__device__ __forceinline__ double scale2(double v, int k)
{
    const long long b = __double_as_longlong(v);
    const int ex = (int)((b >> 52) & 0x7ff);
    if (ex != 0 && ex != 0x7ff && ex + k > 0 && ex + k < 0x7ff) return __longlong_as_double(b + (long long)k * (1LL << 52));
    return v * pow2d(k);
}

// Block = TC_RED_BLOCK consecutive output entries of one (instance,
// timeslice) unit; the unit is the last one whose red0 <= block.  Entry e of
// the unit's output order (B entries [p][...] first, then M entries
// [p][i][k]) is the FP64 sum over site blocks sc = 0, 1, ... of the FP32
// partials part[part_off + sc * n_out + e], times 2^-3s (B) or 2^-2s (M), s
// the timeslice's exponent, written as complex128 or, for complex64 outputs,
// rounded once to FP32.  Each thread owns RED_PER_THREAD entries, TC_RED_BLOCK /
// RED_PER_THREAD apart, and adds each entry's partials in block order.
constexpr int RED_THREADS = 256;
constexpr int RED_PER_THREAD = TC_RED_BLOCK / RED_THREADS;
static_assert(RED_PER_THREAD * RED_THREADS == TC_RED_BLOCK, "reduction block shape");

__global__ void __launch_bounds__(RED_THREADS) reduce_kernel(const InstDev *__restrict__ insts,
                                                             const PsiUnit *__restrict__ units, int n_units,
                                                             long long n_blocks, const unsigned *__restrict__ maxbits,
                                                             const float2 *__restrict__ part)
{
    for (long long blk = blockIdx.x; blk < n_blocks; blk += gridDim.x) {
        int lo = 0, hi = n_units - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (units[mid].red0 <= blk)
                lo = mid;
            else
                hi = mid - 1;
        }
        const PsiUnit un = units[lo];
        const InstDev &I = insts[un.inst];
        const long long nB = I.n_outB, n_out = nB + I.n_outM;
        const long long e0 = (blk - un.red0) * TC_RED_BLOCK + threadIdx.x;
        const float2 *src = part + un.part_off;
        const int n_sc = I.n_sc;
        double re[RED_PER_THREAD], im[RED_PER_THREAD];
#pragma unroll
        for (int q = 0; q < RED_PER_THREAD; q++) {
            const long long e = e0 + q * RED_THREADS;
            const float2 v = e < n_out ? __ldcs(src + e) : make_float2(0.f, 0.f);
            re[q] = widen(v.x);
            im[q] = widen(v.y);
        }
        for (int sc = 1; sc < n_sc; sc++) {
            const float2 *ps = src + (long long)sc * n_out;
            float2 v[RED_PER_THREAD];
#pragma unroll
            for (int q = 0; q < RED_PER_THREAD; q++) {
                const long long e = e0 + q * RED_THREADS;
                v[q] = e < n_out ? __ldcs(ps + e) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int q = 0; q < RED_PER_THREAD; q++) {
                re[q] += widen(v[q].x);
                im[q] += widen(v[q].y);
            }
        }
        const int s = scale_exp(maxbits[I.ts_base + un.t]);
#pragma unroll
        for (int q = 0; q < RED_PER_THREAD; q++) {
            const long long e = e0 + q * RED_THREADS;
            if (e >= n_out) continue;
            long long o;
            int k;
            void *base;
            if (e < nB) {
                base = I.outB;
                o = (long long)un.t * nB + e;
                k = -3 * s;
            } else {
                base = I.outM;
                o = (long long)un.t * I.n_outM + (e - nB);
                k = -2 * s;
            }
            const double vr = scale2(re[q], k), vi = scale2(im[q], k);
            if (I.out_c64)
                reinterpret_cast<float2 *>(base)[o] = make_float2(__double2float_rn(vr), __double2float_rn(vi));
            else
                reinterpret_cast<double2 *>(base)[o] = make_double2(vr, vi);
        }
    }
}

int stage_bytes_for(int max_staged, int nc, bool rd)
{
    const int b = tc_stage_bytes(nc, rd) + max_staged * SLOT_BYTES;
    return (b + 1023) & ~1023;
}

constexpr int SMEM_LIMIT = 227 * 1024;

int smem_for(int ns, int stage_bytes) { return ns * stage_bytes + (int)sizeof(Shared) + 1024; }

template <int ELEM, int TERMS, int NC, bool RD>
cudaError_t launch_one(const InstDev *d_inst, const TileDev *d_tiles, long long n_tiles, const unsigned *maxbits,
                       const uint8_t *psi, float2 *part, unsigned *counter, const TcConfig &cfg, int *status,
                       cudaStream_t s)
{
    KParams kp;
    kp.insts = d_inst;
    kp.tiles = d_tiles;
    kp.maxbits = maxbits;
    kp.psi = psi;
    kp.part = part;
    kp.counter = counter;
    kp.status = status;
    kp.n_tiles = (int)n_tiles;
    kp.chunk_stages = (cfg.chunk_sites * 3) / KSTAGE;
    if (kp.chunk_stages < 1) kp.chunk_stages = 1;
    kp.chunk_stages_b = ((cfg.chunk_sites_b > 0 ? cfg.chunk_sites_b : cfg.chunk_sites) * 3) / KSTAGE;
    if (kp.chunk_stages_b < 1) kp.chunk_stages_b = 1;
    kp.stage_bytes = stage_bytes_for(cfg.max_staged, NC, RD);
    kp.debug_stall = cfg.debug_stall;
    kp.ns = tc_ring_depth(cfg.max_staged, NC, RD);   // deepest stage ring that fits
    if (!kp.ns) return cudaErrorNotSupported;
    const int smem = smem_for(kp.ns, kp.stage_bytes);
    cudaError_t e =
        cudaFuncSetAttribute(tc_kernel<ELEM, TERMS, NC, RD>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int grid = cfg.grid > 0 ? cfg.grid : 148;
    if ((long long)grid > n_tiles) grid = (int)n_tiles;
    tc_kernel<ELEM, TERMS, NC, RD><<<grid, Roles<RD>::NTHREADS, smem, s>>>(kp);
    return cudaGetLastError();
}

template <int NC, bool RD>
void psi_launch(int elem, unsigned grid, const InstDev *d_inst, const PsiUnit *d_units, int n_units, long long n_jobs,
                const unsigned *d_maxbits, uint8_t *psi, cudaStream_t s)
{
    if (elem == 0)
        psi_kernel<0, NC, RD><<<grid, 2 * NC, 0, s>>>(d_inst, d_units, n_units, n_jobs, d_maxbits, psi);
    else
        psi_kernel<1, NC, RD><<<grid, 2 * NC, 0, s>>>(d_inst, d_units, n_units, n_jobs, d_maxbits, psi);
}

}  // namespace

int tc_ring_depth(int max_staged, int ncols, int rows2)
{
    const int sb = stage_bytes_for(max_staged, ncols, rows2 != 0);
    for (int ns = MAX_NS; ns >= 2; ns--)
        if (smem_for(ns, sb) <= SMEM_LIMIT) return ns;
    return 0;
}

bool tc_shape_supported(int ncols, int rows2)
{
    return rows2 ? (ncols == 208 || ncols == 192 || ncols == 176 || ncols == 128)
                 : (ncols == 104 || ncols == 96 || ncols == 80 || ncols == 64);
}

cudaError_t launch_tc(const InstDev *d_inst, const TileDev *d_tiles, long long n_tiles, const unsigned *d_maxbits,
                      const uint8_t *psi, float2 *part, unsigned *counter, const TcConfig &cfg, int *d_status,
                      cudaStream_t s)
{
    if (n_tiles <= 0) return cudaSuccess;
    if (n_tiles > 0x7fffffffLL || cfg.max_staged > TC_MAX_STAGED) return cudaErrorNotSupported;
#define LAPH_TC_CASE(NC, RD)                                                                                    \
    if (cfg.ncols == NC && cfg.rows2 == (RD ? 1 : 0)) {                                                         \
        if (cfg.elem == 0 && cfg.terms == 3)                                                                    \
            return launch_one<0, 3, NC, RD>(d_inst, d_tiles, n_tiles, d_maxbits, psi, part, counter, cfg, d_status, s); \
        if (cfg.elem == 1 && cfg.terms == 3)                                                                    \
            return launch_one<1, 3, NC, RD>(d_inst, d_tiles, n_tiles, d_maxbits, psi, part, counter, cfg, d_status, s); \
        if (cfg.elem == 0 && cfg.terms == 1)                                                                    \
            return launch_one<0, 1, NC, RD>(d_inst, d_tiles, n_tiles, d_maxbits, psi, part, counter, cfg, d_status, s); \
        if (cfg.elem == 1 && cfg.terms == 1)                                                                    \
            return launch_one<1, 1, NC, RD>(d_inst, d_tiles, n_tiles, d_maxbits, psi, part, counter, cfg, d_status, s); \
    }
    LAPH_TC_CASE(104, false)
    LAPH_TC_CASE(96, false)
    LAPH_TC_CASE(80, false)
    LAPH_TC_CASE(64, false)
    LAPH_TC_CASE(208, true)
    LAPH_TC_CASE(192, true)
    LAPH_TC_CASE(176, true)
    LAPH_TC_CASE(128, true)
#undef LAPH_TC_CASE
    return cudaErrorNotSupported;
}

cudaError_t launch_reduce(const InstDev *d_inst, const PsiUnit *d_units, int n_units, long long n_blocks,
                          const unsigned *d_maxbits, const float2 *part, cudaStream_t s)
{
    if (n_blocks <= 0 || n_units <= 0) return cudaSuccess;
    const long long grid = n_blocks < (1LL << 20) ? n_blocks : (1LL << 20);
    reduce_kernel<<<(unsigned)grid, RED_THREADS, 0, s>>>(d_inst, d_units, n_units, n_blocks, d_maxbits, part);
    return cudaGetLastError();
}

cudaError_t launch_psi(const InstDev *d_inst, const PsiUnit *d_units, int n_units, long long n_jobs,
                       const unsigned *d_maxbits, int elem, int ncols, int rows2, uint8_t *psi, cudaStream_t s)
{
    if (n_jobs <= 0 || n_units <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)(n_jobs < (1LL << 20) ? n_jobs : (1LL << 20));
    if (!rows2 && ncols == 104)
        psi_launch<104, false>(elem, grid, d_inst, d_units, n_units, n_jobs, d_maxbits, psi, s);
    else if (!rows2 && ncols == 96)
        psi_launch<96, false>(elem, grid, d_inst, d_units, n_units, n_jobs, d_maxbits, psi, s);
    else if (!rows2 && ncols == 80)
        psi_launch<80, false>(elem, grid, d_inst, d_units, n_units, n_jobs, d_maxbits, psi, s);
    else if (!rows2 && ncols == 64)
        psi_launch<64, false>(elem, grid, d_inst, d_units, n_units, n_jobs, d_maxbits, psi, s);
    else if (rows2 && ncols == 208)
        psi_launch<208, true>(elem, grid, d_inst, d_units, n_units, n_jobs, d_maxbits, psi, s);
    else if (rows2 && ncols == 192)
        psi_launch<192, true>(elem, grid, d_inst, d_units, n_units, n_jobs, d_maxbits, psi, s);
    else if (rows2 && ncols == 176)
        psi_launch<176, true>(elem, grid, d_inst, d_units, n_units, n_jobs, d_maxbits, psi, s);
    else if (rows2 && ncols == 128)
        psi_launch<128, true>(elem, grid, d_inst, d_units, n_units, n_jobs, d_maxbits, psi, s);
    else
        return cudaErrorNotSupported;
    return cudaGetLastError();
}

}  // namespace laph
