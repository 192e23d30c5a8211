// tcgen05 tensor-core path of the block contraction (K-b..K-f fused, K-i).
//
// Same decomposition as the FP32 path: rows are meson rows (A = conj(phi_i))
// and diquark rows (A = phi_i x phi_j, i<j, colex order), columns are (k,p)
// with Psi = ph_p(x) phi_k, and the complex product runs over K = 3V
// (site, colour):  C[row][col] = sum A(x,c) Psi(x,c).
//
// Complex -> real embedding (no extra flops): A is stored as interleaved
// (re, im) along K; every complex column becomes two real B rows,
//   re-row [Psi_re, -Psi_im]  ->  C_re,    im-row [Psi_im, Psi_re]  ->  C_im.
//
// Precision: phi is rescaled by an exact power of two per timeslice, every
// operand value v is split into hi = RN16(v), lo = RN16(v - hi) (FP16 or
// BF16), and the tensor core accumulates hi*hi + hi*lo + lo*hi in FP32 (one
// term, hi*hi, in the plain modes).  The FP32 accumulator in tensor memory is
// drained every `chunk_stages` K stages and added in FP64 (after undoing the
// scale) into the complex128 output, which each element's owner alone
// touches.
//
// CTA organisation (persistent, one CTA per SM, dynamic tile scheduler):
//   warps 0-3   A producers: one TMEM lane (tile row) per thread; compute the
//               row's 32 K entries of a stage in registers and tcgen05.st
//               them (hi and lo) into a tensor-memory stage slot;
//   warps 4-7   B producers: one complex column per thread; compute Psi and
//               store both real rows (hi and lo) into shared memory in the
//               128-byte-swizzled K-major layout the MMA descriptor reads;
//   warps 8-11  epilogue: tcgen05.ld of the accumulator, FP64 reduction;
//   warp 12     TMEM allocation and the single-thread MMA issue
//               (tcgen05.mma kind::f16, A from TMEM, B from SMEM, M=128,
//               N = 2 * columns <= 256, K = 16 per instruction);
//   warp 13     tile scheduler (global atomic counter -> 2-slot ring).
// Every wait on an mbarrier is bounded; on expiry the CTA records
// STATUS_TIMEOUT, raises a shared abort flag and all roles return.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "laph_internal.cuh"

namespace laph {
namespace {

constexpr int NTHREADS = 448;
constexpr int WARP_B0 = 4;
constexpr int WARP_E0 = 8;
constexpr int WARP_MMA = 12;
constexpr int WARP_SCHED = 13;
constexpr int NA = 4;                       // A stage slots in tensor memory
constexpr int NB = 3;                       // B stage buffers in shared memory
constexpr int KSTAGE = 32;                  // complex K entries per stage (= 64 real)
constexpr int B_ROWS = 2 * TC_TC;           // real B rows per tile (256)
constexpr int B_BYTES = B_ROWS * 128;       // one of hi/lo: 256 rows x 64 halves
constexpr int STAGE_BYTES = 2 * B_BYTES;    // hi + lo
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t A_SLOT_COLS = 64;        // 32 columns hi + 32 columns lo
constexpr uint32_t ACC_COL = NA * A_SLOT_COLS;  // accumulator at columns [256, 512)
constexpr long long WAIT_LIMIT = 4000000000LL;  // cycles (about 2 s at the top clock)
constexpr int N_CONSUMER_WARPS = 13;         // warps that read a tile slot

static_assert(TC_TR == 128 && TC_TC == 128, "layout assumes 128 x 128 tiles");
static_assert(ACC_COL + 2 * TC_TC <= TMEM_COLS, "tensor memory budget");

struct Shared {
    uint64_t a_full[NA], a_empty[NA];
    uint64_t b_full[NB], b_empty[NB];
    uint64_t acc_full, acc_empty;
    uint64_t tile_full[2], tile_empty[2];
    uint64_t done;
    int tile_id[2];
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

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]),
        "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]),
        "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
        : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
          "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
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

__device__ __forceinline__ float2 ldg2(const float2 *p) { return __ldg(p); }

// ------------------------------------------------------------ waits

struct Ctx {
    Shared *S;
    int *status;
    int lane;
};

// Warp-wide bounded wait (every lane calls it; the result is warp-uniform).
__device__ __forceinline__ bool warp_wait(const Ctx &c, uint64_t *bar, uint32_t parity)
{
    long long t0 = 0;
    bool started = false;
    while (true) {
        const bool ok = mbar_try_wait(bar, parity);
        if (__all_sync(0xffffffffu, ok)) return true;
        const int ab = *(volatile int *)&c.S->abort;
        if (__any_sync(0xffffffffu, ab != 0)) return false;
        if (!started) {
            t0 = clock64();
            started = true;
        } else {
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
}

// Single-thread bounded wait.
__device__ __forceinline__ bool thread_wait(const Ctx &c, uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*(volatile int *)&c.S->abort) return false;
        if (clock64() - t0 > WAIT_LIMIT) {
            *(volatile int *)&c.S->abort = 1;
            atomicOr(c.status, STATUS_TIMEOUT);
            return false;
        }
    }
}

// Next tile id from the scheduler ring (warp-wide); -1 = no more, -2 = abort.
__device__ __forceinline__ int next_tile(const Ctx &c, int it)
{
    const int s = it & 1;
    const uint32_t ph = (uint32_t)(it >> 1) & 1u;
    if (!warp_wait(c, &c.S->tile_full[s], ph)) return -2;
    const int id = *(volatile int *)&c.S->tile_id[s];
    __syncwarp();
    if (c.lane == 0) mbar_arrive(&c.S->tile_empty[s]);
    return id;
}

// ------------------------------------------------------------ producers

// Diquark entries of one stage for a pair row: K-local index kl = 3*xs + c - R0
// for the sites x0 + xs (R0 = kappa0 mod 3), scaled by sc2 and split.
template <int ELEM, int R0>
__device__ __forceinline__ void diquark_stage(const float2 *__restrict__ pi, const float2 *__restrict__ pj,
                                              long long x0, long long V, float sc2, uint32_t (&hi)[32],
                                              uint32_t (&lo)[32])
{
#pragma unroll
    for (int xs = 0; xs < 12; xs++) {
        if (3 * xs - R0 > KSTAGE - 1) break;
        const long long x = x0 + xs;
        float2 u[3], v[3];
        if (x < V) {
#pragma unroll
            for (int a = 0; a < 3; a++) {
                u[a] = ldg2(pi + 3 * x + a);
                v[a] = ldg2(pj + 3 * x + a);
            }
        } else {
#pragma unroll
            for (int a = 0; a < 3; a++) u[a] = v[a] = make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const int kl = 3 * xs + c - R0;
            if (kl < 0 || kl >= KSTAGE) continue;
            const float2 d = cross_c(u, v, c);
            split2<ELEM>(d.x * sc2, d.y * sc2, hi[kl], lo[kl]);
        }
    }
}

template <int ELEM>
__device__ __forceinline__ void produce_a_stage(int kind, const float2 *__restrict__ pi, const float2 *__restrict__ pj,
                                                long long kap0, long long V, float sc, uint32_t (&hi)[32],
                                                uint32_t (&lo)[32])
{
    const long long K = 3 * V;
    if (kind == 2) {  // diquark row
        const long long x0 = kap0 / 3;
        const int r0 = (int)(kap0 - 3 * x0);
        const float sc2 = sc * sc;
        if (r0 == 0)
            diquark_stage<ELEM, 0>(pi, pj, x0, V, sc2, hi, lo);
        else if (r0 == 1)
            diquark_stage<ELEM, 1>(pi, pj, x0, V, sc2, hi, lo);
        else
            diquark_stage<ELEM, 2>(pi, pj, x0, V, sc2, hi, lo);
    } else if (kind == 1) {  // meson row: conj(phi_i)
#pragma unroll
        for (int kl = 0; kl < KSTAGE; kl++) {
            const long long kap = kap0 + kl;
            float2 a = make_float2(0.f, 0.f);
            if (kap < K) a = ldg2(pi + kap);
            split2<ELEM>(a.x * sc, -a.y * sc, hi[kl], lo[kl]);
        }
    } else {
#pragma unroll
        for (int kl = 0; kl < KSTAGE; kl++) hi[kl] = lo[kl] = 0u;
    }
}

// ------------------------------------------------------------ the kernel

template <int ELEM, int TERMS>
__global__ void __launch_bounds__(NTHREADS, 1)
tc_kernel(const InstDev *__restrict__ insts, const TileDev *__restrict__ tiles, int n_tiles,
          const unsigned *__restrict__ maxbits, unsigned long long *__restrict__ counter, int chunk_stages,
          int debug_stall, int *__restrict__ status)
{
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *bstage = smem;
    Shared *S = reinterpret_cast<Shared *>(smem + NB * STAGE_BYTES);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Ctx c{S, status, lane};

    if (threadIdx.x == 0) {
        for (int s = 0; s < NA; s++) {
            mbar_init(&S->a_full[s], 4);
            mbar_init(&S->a_empty[s], 1);
        }
        for (int s = 0; s < NB; s++) {
            mbar_init(&S->b_full[s], 4);
            mbar_init(&S->b_empty[s], 1);
        }
        mbar_init(&S->acc_full, 1);
        mbar_init(&S->acc_empty, 4);
        for (int s = 0; s < 2; s++) {
            mbar_init(&S->tile_full[s], 1);
            mbar_init(&S->tile_empty[s], N_CONSUMER_WARPS);
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

    if (warp == WARP_SCHED) {
        // ---------------------------------------------------------- scheduler
        if (lane == 0) {
            for (int it = 0;; it++) {
                const int s = it & 1;
                const uint32_t ph = (uint32_t)(it >> 1) & 1u;
                if (!thread_wait(c, &S->tile_empty[s], ph ^ 1u)) break;
                const unsigned long long id = atomicAdd(counter, 1ULL);
                const int v = id < (unsigned long long)n_tiles ? (int)id : -1;
                *(volatile int *)&S->tile_id[s] = v;
                mbar_arrive(&S->tile_full[s]);
                if (v < 0) break;
            }
        }
    } else if (warp < WARP_B0) {
        // ---------------------------------------------------------- A producers
        const int quad = warp & 3;
        const int r = quad * 32 + lane;
        const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
        uint32_t gs = 0;
        bool stalled = false;
        for (int it = 0;; it++) {
            const int id = next_tile(c, it);
            if (id < 0) break;
            const TileDev td = tiles[id];
            const InstDev &I = insts[td.inst];
            const long long V = I.V;
            const int g = td.row0 + r;
            int kind = 0, vi = 0, vj = 0;
            if (g < I.rows) {
                if (g < I.mes_rows) {
                    kind = 1;
                    vi = g;
                } else {
                    kind = 2;
                    pair_of(g - I.mes_rows, vi, vj);
                }
            }
            const float sc = pow2f(scale_exp(maxbits[I.ts_base + td.t]));
            const float2 *pi = I.phi + ((long long)td.t * I.N + vi) * V * 3;
            const float2 *pj = I.phi + ((long long)td.t * I.N + vj) * V * 3;
            const int n_st = (int)((3 * V + KSTAGE - 1) / KSTAGE);
            bool ok = true;
            for (int st = 0; st < n_st; st++, gs++) {
                const int slot = gs % NA;
                const uint32_t ph = (gs / NA) & 1u;
                if (!warp_wait(c, &S->a_empty[slot], ph ^ 1u)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                uint32_t hi[32], lo[32];
                produce_a_stage<ELEM>(kind, pi, pj, (long long)st * KSTAGE, V, sc, hi, lo);
                const uint32_t ta = tmem + lane_base + (uint32_t)slot * A_SLOT_COLS;
                tmem_st32(ta, hi);
                tmem_st32(ta + 32, lo);
                tmem_wait_st();
                tc_fence_before();
                __syncwarp();
                const bool skip = debug_stall && !stalled && blockIdx.x == 0 && warp == 0;
                if (skip) stalled = true;
                if (lane == 0 && !skip) mbar_arrive(&S->a_full[slot]);
            }
            if (!ok) break;
        }
    } else if (warp < WARP_E0) {
        // ---------------------------------------------------------- B producers
        const int cl = (warp - WARP_B0) * 32 + lane;  // complex column within the tile
        uint32_t gs = 0;
        for (int it = 0;; it++) {
            const int id = next_tile(c, it);
            if (id < 0) break;
            const TileDev td = tiles[id];
            const InstDev &I = insts[td.inst];
            const long long V = I.V, K = 3 * V;
            const int ncols = min(TC_TC, I.cols - td.col0);
            const int ncols_pad = (ncols + 7) & ~7;
            const bool valid = cl < ncols;
            const bool write = cl < ncols_pad;
            int k = 0, p = 0;
            if (valid) {
                k = (td.col0 + cl) / I.P;
                p = td.col0 + cl - k * I.P;
            }
            const float sc = pow2f(scale_exp(maxbits[I.ts_base + td.t]));
            const float2 *pk = I.phi + ((long long)td.t * I.N + k) * V * 3;
            const float2 *php = I.phase + (long long)p * V;
            const int n_st = (int)((K + KSTAGE - 1) / KSTAGE);
            const int n0 = 2 * cl, n1 = 2 * cl + 1;
            bool ok = true;
            for (int st = 0; st < n_st; st++, gs++) {
                const int slot = gs % NB;
                const uint32_t ph = (gs / NB) & 1u;
                if (!warp_wait(c, &S->b_empty[slot], ph ^ 1u)) {
                    ok = false;
                    break;
                }
                if (write) {
                    uint8_t *bhi = bstage + slot * STAGE_BYTES;
                    uint8_t *blo = bhi + B_BYTES;
                    const long long kap0 = (long long)st * KSTAGE;
#pragma unroll
                    for (int j = 0; j < 8; j++) {
                        uint32_t rh[4], rl[4], ih[4], il[4];
#pragma unroll
                        for (int u = 0; u < 4; u++) {
                            const long long kap = kap0 + 4 * j + u;
                            float2 psi = make_float2(0.f, 0.f);
                            if (valid && kap < K) {
                                const float2 f = ldg2(pk + kap);
                                const float2 e = ldg2(php + kap / 3);
                                psi = cmulf(e, f);
                            }
                            uint32_t h, l;
                            split2<ELEM>(psi.x * sc, psi.y * sc, h, l);
                            rh[u] = h ^ 0x80000000u;           // (re, -im)
                            rl[u] = l ^ 0x80000000u;
                            ih[u] = __byte_perm(h, 0, 0x1032);  // (im, re)
                            il[u] = __byte_perm(l, 0, 0x1032);
                        }
                        *reinterpret_cast<uint4 *>(bhi + swz(n0, j)) = make_uint4(rh[0], rh[1], rh[2], rh[3]);
                        *reinterpret_cast<uint4 *>(bhi + swz(n1, j)) = make_uint4(ih[0], ih[1], ih[2], ih[3]);
                        *reinterpret_cast<uint4 *>(blo + swz(n0, j)) = make_uint4(rl[0], rl[1], rl[2], rl[3]);
                        *reinterpret_cast<uint4 *>(blo + swz(n1, j)) = make_uint4(il[0], il[1], il[2], il[3]);
                    }
                }
                fence_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&S->b_full[slot]);
            }
            if (!ok) break;
        }
    } else if (warp < WARP_MMA) {
        // ---------------------------------------------------------- epilogue
        const int quad = warp & 3;
        const int r = quad * 32 + lane;
        const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
        uint32_t gc = 0;
        for (int it = 0;; it++) {
            const int id = next_tile(c, it);
            if (id < 0) break;
            const TileDev td = tiles[id];
            const InstDev &I = insts[td.inst];
            const long long V = I.V;
            const int ncols = min(TC_TC, I.cols - td.col0);
            const int n_real = 2 * ((ncols + 7) & ~7);
            const int g = td.row0 + r;
            const bool rvalid = g < I.rows;
            const bool meson = g < I.mes_rows;
            int pi_ = 0, pj_ = 0;
            long long q = 0;
            if (rvalid && !meson) {
                q = g - I.mes_rows;
                pair_of(q, pi_, pj_);
            }
            const int s = scale_exp(maxbits[I.ts_base + td.t]);
            const double fac = meson ? pow2d(-2 * s) : pow2d(-3 * s);
            const int n_st = (int)((3 * V + KSTAGE - 1) / KSTAGE);
            const int n_ch = (n_st + chunk_stages - 1) / chunk_stages;
            const long long tP = (long long)td.t * I.P;
            bool ok = true;
            for (int ch = 0; ch < n_ch; ch++, gc++) {
                if (!warp_wait(c, &S->acc_full, gc & 1u)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                for (int b = 0; b * 32 < n_real; b++) {
                    uint32_t v[32];
                    tmem_ld32(tmem + lane_base + ACC_COL + 32u * b, v);
                    tmem_wait_ld();
#pragma unroll
                    for (int u = 0; u < 16; u++) {
                        const int cc = 16 * b + u;
                        if (!rvalid || cc >= ncols) continue;
                        const int col = td.col0 + cc;
                        const int k = col / I.P, p = col - k * I.P;
                        double2 *dst;
                        if (meson) {
                            dst = I.outM + ((tP + p) * I.N + g) * I.N + k;
                        } else {
                            if (k <= pj_) continue;
                            dst = I.outB + (tP + p) * I.n_trip + binom3(k) + q;
                        }
                        double2 val = make_double2((double)__uint_as_float(v[2 * u]) * fac,
                                                   (double)__uint_as_float(v[2 * u + 1]) * fac);
                        if (ch > 0) {
                            const double2 old = *dst;
                            val.x += old.x;
                            val.y += old.y;
                        }
                        *dst = val;
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&S->acc_empty);
            }
            if (!ok) break;
        }
    } else {
        // ---------------------------------------------------------- MMA issue
        uint32_t ga = 0, gb = 0, gc = 0;
        bool issued = false;
        for (int it = 0;; it++) {
            const int id = next_tile(c, it);
            if (id < 0) break;
            const TileDev td = tiles[id];
            const InstDev &I = insts[td.inst];
            const long long V = I.V;
            const int ncols = min(TC_TC, I.cols - td.col0);
            const int n_real = 2 * ((ncols + 7) & ~7);
            const uint32_t idesc = idesc_f16(n_real, ELEM);
            const int n_st = (int)((3 * V + KSTAGE - 1) / KSTAGE);
            bool ok = true;
            for (int st = 0; st < n_st; st++) {
                const bool chunk_start = (st % chunk_stages) == 0;
                const bool chunk_end = ((st + 1) % chunk_stages) == 0 || st + 1 == n_st;
                if (chunk_start) {
                    if (!warp_wait(c, &S->acc_empty, (gc & 1u) ^ 1u)) {
                        ok = false;
                        break;
                    }
                }
                const int sa = ga % NA, sb = gb % NB;
                if (!warp_wait(c, &S->a_full[sa], (ga / NA) & 1u) || !warp_wait(c, &S->b_full[sb], (gb / NB) & 1u)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                if (lane == 0) {
                    const uint32_t a_hi = tmem + (uint32_t)sa * A_SLOT_COLS, a_lo = a_hi + 32;
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
                ga++;
                gb++;
                if (chunk_end) gc++;
            }
            if (!ok) break;
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

template <int ELEM, int TERMS>
cudaError_t launch_one(const InstDev *d_inst, const TileDev *d_tiles, long long n_tiles, const unsigned *maxbits,
                       unsigned long long *counter, const TcConfig &cfg, int *status, cudaStream_t s)
{
    const int smem = NB * STAGE_BYTES + (int)sizeof(Shared) + 1024;
    cudaError_t e = cudaFuncSetAttribute(tc_kernel<ELEM, TERMS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int grid = cfg.grid > 0 ? cfg.grid : 148;
    if ((long long)grid > n_tiles) grid = (int)n_tiles;
    int chunk_stages = (cfg.chunk_sites * 3) / KSTAGE;
    if (chunk_stages < 1) chunk_stages = 1;
    tc_kernel<ELEM, TERMS><<<grid, NTHREADS, smem, s>>>(d_inst, d_tiles, (int)n_tiles, maxbits, counter, chunk_stages,
                                                      cfg.debug_stall, status);
    return cudaGetLastError();
}

}  // namespace

int tc_smem_bytes() { return NB * STAGE_BYTES + (int)sizeof(Shared) + 1024; }

cudaError_t launch_tc(const InstDev *d_inst, const TileDev *d_tiles, long long n_tiles, const unsigned *d_maxbits,
                      unsigned long long *d_counter, const TcConfig &cfg, int *d_status, cudaStream_t s)
{
    if (n_tiles <= 0) return cudaSuccess;
    if (n_tiles > 0x7fffffffLL) return cudaErrorNotSupported;
    if (cfg.elem == 0 && cfg.terms == 3) return launch_one<0, 3>(d_inst, d_tiles, n_tiles, d_maxbits, d_counter, cfg, d_status, s);
    if (cfg.elem == 1 && cfg.terms == 3) return launch_one<1, 3>(d_inst, d_tiles, n_tiles, d_maxbits, d_counter, cfg, d_status, s);
    if (cfg.elem == 0 && cfg.terms == 1) return launch_one<0, 1>(d_inst, d_tiles, n_tiles, d_maxbits, d_counter, cfg, d_status, s);
    if (cfg.elem == 1 && cfg.terms == 1) return launch_one<1, 1>(d_inst, d_tiles, n_tiles, d_maxbits, d_counter, cfg, d_status, s);
    return cudaErrorNotSupported;
}

}  // namespace laph
