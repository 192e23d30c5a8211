// laph_blocks_noalloc: the FP32 block contraction for callers that cannot
// allocate device memory.
//
// Some callers may not call cudaMalloc or any allocating routine: code that
// runs where device allocation is forbidden or unsafe (inside a host callback
// or a real-time loop that must not block on the allocator, or an embedding
// framework that owns the device memory pool and rejects foreign
// allocations).  This entry point serves them: the caller passes only its
// inputs and outputs, and every piece of scratch the computation needs (the
// instance descriptor, the momenta, the tile table and the FP32 phase table)
// lives in one file-scope device array of fixed size, which exists on every
// GPU that loads the library until the process exits.
//
// The array is shared by all calls and keeps the last call's contents; each
// call rewrites every byte it reads before reading it, so nothing has to
// start at zero.  Calls whose work overlaps on the GPU (different streams, or
// different host threads, without ordering between them) race on the array.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>
#include <vector>

#include "laph.h"
#include "laph_internal.cuh"

namespace laph {
namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)LAPH_NOALLOC_SCRATCH_BYTES;
constexpr int NOALLOC_MAX_MOM = 64;
constexpr int NOALLOC_MAX_ROW_TILES = 4096;
// the public header states the scratch use of one tile record
static_assert(sizeof(TileDev) == 72, "the documented tile-record size in laph.h");

// The scratch array.  Host code must not pass its name to a kernel: on the
// host it is only a stand-in symbol; its device address is obtained with
// cudaGetSymbolAddress (see scratch_on_current_device).
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// The array's device address is a property of the CUDA context it was
// loaded into.  It is looked up once per context -- in the normal case once
// per device, in the device's primary context -- and cached under the
// context's unique ID, so that a context created after a device reset (or a
// context the caller made current through the driver API) gets its own
// lookup instead of a stale address.
struct ScratchAddr {
    unsigned long long ctx_id;
    void *addr;
};
std::mutex g_setup_mutex;
std::vector<ScratchAddr> g_scratch_addr;

// Driver functions reached through the runtime (so that the library itself
// loads on a host without the driver, e.g. to be inspected).
PFN_cuCtxGetCurrent_v4000 g_ctx_current = nullptr;
PFN_cuCtxGetId_v12000 g_ctx_id = nullptr;

// ID of the current context, after the runtime has made one current.
cudaError_t current_context_id(unsigned long long *id)
{
    cudaError_t e;
    if (!g_ctx_current || !g_ctx_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = cudaDriverEntryPointSymbolNotFound;
        if ((e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 4000, cudaEnableDefault, &q1)) != cudaSuccess)
            return e;
        if ((e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2)) != cudaSuccess)
            return e;
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return cudaErrorNotSupported;
        g_ctx_current = (PFN_cuCtxGetCurrent_v4000)f1;
        g_ctx_id = (PFN_cuCtxGetId_v12000)f2;
    }
    CUcontext ctx = nullptr;
    if (g_ctx_current(&ctx) != CUDA_SUCCESS) return cudaErrorInitializationError;
    if (!ctx) {
        // no context yet on this thread: the lookup below initialises the
        // current device's primary context and makes it current
        void *p = nullptr;
        if ((e = cudaGetSymbolAddress(&p, g_noalloc_scratch)) != cudaSuccess) return e;
        if (g_ctx_current(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorInitializationError;
    }
    return g_ctx_id(ctx, id) == CUDA_SUCCESS ? cudaSuccess : cudaErrorInitializationError;
}

// Device address of the scratch array in the current context (the first call
// in a context looks it up, so it must not be made while a stream is being
// captured).
cudaError_t scratch_on_current_device(unsigned char **addr)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    unsigned long long id = 0;
    cudaError_t e = current_context_id(&id);
    if (e != cudaSuccess) return e;
    for (const ScratchAddr &a : g_scratch_addr)
        if (a.ctx_id == id) {
            *addr = (unsigned char *)a.addr;
            return cudaSuccess;
        }
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr.push_back(ScratchAddr{id, p});
    *addr = (unsigned char *)p;
    return cudaSuccess;
}

struct NoallocSetup {
    InstDev inst;          // pointers to phi, outputs and the phase table already filled
    int32_t mom[3 * NOALLOC_MAX_MOM];
    int n_row_tiles;
    int tiles_per_ts;
};

// Needed column tiles of FP32-path row tile rt (same rule as the plan's tile table).
__host__ __device__ inline int simt_cols_needed(const InstDev &d, int rt)
{
    const int row0 = rt * SIMT_TR;
    int jmin = -1;
    if (row0 >= d.mes_rows) {
        int i, j;
        pair_of(row0 - d.mes_rows, i, j);
        jmin = j;
    }
    int count = 0;
    for (int col0 = 0; col0 < d.cols; col0 += SIMT_TC) {
        const int nc = d.cols - col0 < SIMT_TC ? d.cols - col0 : SIMT_TC;
        const int kmax = (col0 + nc - 1) / d.P;
        if (jmin >= 0 && kmax <= jmin) continue;
        count++;
    }
    return count;
}

// One block: writes the descriptor and momenta into the scratch, counts the
// tiles of every row tile, scans the counts and writes the tile table for
// all timeslices.
__global__ void noalloc_setup_kernel(NoallocSetup su, InstDev *d_inst, int32_t *d_mom, int *d_off, TileDev *d_tiles)
{
    const InstDev &d = su.inst;
    if (threadIdx.x == 0) *d_inst = d;
    for (int q = threadIdx.x; q < 3 * d.P; q += blockDim.x) d_mom[q] = su.mom[q];
    for (int rt = threadIdx.x; rt < su.n_row_tiles; rt += blockDim.x) d_off[rt] = simt_cols_needed(d, rt);
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int rt = 0; rt < su.n_row_tiles; rt++) {
            const int c = d_off[rt];
            d_off[rt] = acc;
            acc += c;
        }
    }
    __syncthreads();
    for (int rt = threadIdx.x; rt < su.n_row_tiles; rt += blockDim.x) {
        const int row0 = rt * SIMT_TR;
        int jmin = -1;
        if (row0 >= d.mes_rows) {
            int i, j;
            pair_of(row0 - d.mes_rows, i, j);
            jmin = j;
        }
        int k = d_off[rt];
        for (int col0 = 0; col0 < d.cols; col0 += SIMT_TC) {
            const int nc = d.cols - col0 < SIMT_TC ? d.cols - col0 : SIMT_TC;
            const int kmax = (col0 + nc - 1) / d.P;
            if (jmin >= 0 && kmax <= jmin) continue;
            for (int t = 0; t < d.T; t++) {
                TileDev u{0, t, row0, col0, 0, 0, 0, 0, 0, 0, nc, 0, 0};
                d_tiles[(long long)t * su.tiles_per_ts + k] = u;
            }
            k++;
        }
    }
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace
}  // namespace laph

using laph::InstDev;
using laph::TileDev;

extern "C" int laph_blocks_noalloc(const void *phi, int L, int T, int N, const int32_t *momenta, int n_mom, void *out_B,
                                   void *out_M, void *stream)
{
    if (!phi || !momenta || (!out_B && !out_M)) return LAPH_ERR_ARG;
    if (L < 1 || L > 512 || T < 1 || N < 1 || N > 4096 || n_mom < 1 || n_mom > laph::NOALLOC_MAX_MOM) return LAPH_ERR_ARG;
    if (out_B && N < 3) return LAPH_ERR_ARG;
    if ((long long)N > 3LL * L * L * L) return LAPH_ERR_ARG;
    if (((uintptr_t)phi) % 8 || (out_B && ((uintptr_t)out_B) % 16) || (out_M && ((uintptr_t)out_M) % 16))
        return LAPH_ERR_ARG;
    for (int q = 0; q < 3 * n_mom; q++)
        if (momenta[q] > (1 << 20) || momenta[q] < -(1 << 20)) return LAPH_ERR_ARG;

    // descriptor of the single instance (host copy, passed by value)
    laph::NoallocSetup su;
    memset(&su, 0, sizeof(su));
    InstDev &d = su.inst;
    d.phi = (const float2 *)phi;
    d.phi_u = d.phi_v = d.phi;
    d.blkv_off = -1;
    d.n_fields = 1;
    d.Nc = N;
    d.outB = (double2 *)out_B;
    d.outM = (double2 *)out_M;
    d.L = L;
    d.T = T;
    d.N = N;
    d.P = n_mom;
    d.V = (long long)L * L * L;
    d.Vs = d.V + (d.V & 1);
    d.n_trip = laph::binom3(N);
    d.blk_off = -1;
    d.mes_rows = out_M ? N : 0;
    d.pair_rows = out_B ? (int)laph::binom2(N) : 0;
    d.rows = d.mes_rows + d.pair_rows;
    d.cols = N * n_mom;
    for (int q = 0; q < 3 * n_mom; q++) su.mom[q] = momenta[q];

    // sizes, checked against the fixed scratch array before anything runs
    const int n_row_tiles = (d.rows + laph::SIMT_TR - 1) / laph::SIMT_TR;
    if (n_row_tiles > laph::NOALLOC_MAX_ROW_TILES) return LAPH_ERR_WORKSPACE;
    long long per_ts = 0;
    for (int rt = 0; rt < n_row_tiles; rt++) per_ts += laph::simt_cols_needed(d, rt);
    const long long n_tiles = per_ts * T;
    su.n_row_tiles = n_row_tiles;
    su.tiles_per_ts = (int)per_ts;
    const size_t off_inst = 0;
    const size_t off_mom = laph::align256(sizeof(InstDev));
    const size_t off_cnt = off_mom + laph::align256(sizeof(int32_t) * 3 * n_mom);
    const size_t off_tiles = off_cnt + laph::align256(sizeof(int) * n_row_tiles);
    const size_t off_phase = off_tiles + laph::align256(sizeof(TileDev) * (size_t)n_tiles);
    const size_t need = off_phase + laph::align256(sizeof(float2) * (size_t)n_mom * (size_t)d.Vs);
    if (need > laph::NOALLOC_SCRATCH_BYTES) return LAPH_ERR_WORKSPACE;

    unsigned char *scratch = nullptr;
    cudaError_t e = laph::scratch_on_current_device(&scratch);
    if (e != cudaSuccess) return LAPH_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    InstDev *d_inst = (InstDev *)(scratch + off_inst);
    int32_t *d_mom = (int32_t *)(scratch + off_mom);
    int *d_cnt = (int *)(scratch + off_cnt);
    TileDev *d_tiles = (TileDev *)(scratch + off_tiles);
    float2 *d_phase = (float2 *)(scratch + off_phase);
    d.phase = d_phase;

    laph::noalloc_setup_kernel<<<1, 256, 0, s>>>(su, d_inst, d_mom, d_cnt, d_tiles);
    if ((e = cudaGetLastError()) != cudaSuccess) return LAPH_ERR_CUDA;
    if ((e = laph::launch_phase_table(L, d_mom, n_mom, nullptr, d_phase, s)) != cudaSuccess) return LAPH_ERR_CUDA;
    laph::SimtConfig cfg;
    cfg.chunk_sites = 1024;
    if ((e = laph::launch_simt(d_inst, d_tiles, n_tiles, cfg, nullptr, s)) != cudaSuccess) return LAPH_ERR_CUDA;
    return LAPH_OK;
}
