// Internal declarations shared by the CUDA translation units of the LapH
// block library.  Not part of the public ABI (that is include/laph.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace laph {

// Device status bits (OR-ed into the plan's status word).
constexpr int STATUS_TIMEOUT = 1;
constexpr int STATUS_CHECK = 2;

// Kinds of instance.  INST_BLOCKS: the LapH meson and baryon blocks of one
// set of vectors phi (B packed over i<j<k).  INST_TRIPLETS: three-field
// triplets B3[p][i][j][k] = sum_x ph eps phi_i psi_j chi_k, dense.
// INST_DOUBLETS: two-field doublets M2[p][i][j] = sum_x ph conj(phi_i) psi_j.
constexpr int INST_BLOCKS = 0;
constexpr int INST_TRIPLETS = 1;
constexpr int INST_DOUBLETS = 2;

// One instance of a batch, as the kernels see it.  Row space of the
// contraction: rows [0, mes_rows) are meson rows (vector i = row, A operand
// conj(phi_u_i)), rows [mes_rows, mes_rows + pair_rows) are diquark rows
// (A operand phi_u_i x phi_v_j): pair q = row - mes_rows in colex order
// q = C(j,2) + i for INST_BLOCKS, q = i * N + j for INST_TRIPLETS.  Column
// space: col = k * P + p, k < Nc, B operand ph_p * phi_k (phi is the column
// field, of Nc vectors; the row fields have N).
struct InstDev {
    const float2 *phi;       // [T][N][V][3] column field (phi; chi for triplets, psi for doublets)
    const float2 *phi_u;     // [T][N][V][3] first row field (phi)
    const float2 *phi_v;     // [T][N][V][3] second row field (phi; psi for triplets)
    double2 *outB;           // [T][P][C(N,3)] (float2 entries when out_c64)
    double2 *outM;           // [T][P][N][N] (float2 entries when out_c64)
    const float2 *phase;     // [P][Vs], FP32 rounding of the FP64 phase
    float2 *phi_blk;         // tensor-core path: scaled, site-blocked copy of phi_u in the workspace
    float2 *blk_v;           // the same for phi_v (triplets only)
    long long V;
    long long Vs;            // V rounded up to even: row stride of `phase`
    long long n_trip;        // C(N,3)
    long long blk_off;       // byte offset of phi_blk in the workspace (-1: none)
    long long blkv_off;      // byte offset of blk_v in the workspace (-1: none)
    int L, T, N, P;
    int mes_rows;            // N, or 0 when mesons are skipped
    int pair_rows;           // C(N,2), or 0 when baryons are skipped
    int rows;                // mes_rows + pair_rows
    int cols;                // N * P
    int ts_base;             // index of (this instance, t = 0) among all timeslices of the batch
    int nblk;                // site blocks: ceil(V / TC_BS)
    int n_ct;                // column tiles of the tensor-core path: ceil(cols / the plan's tile width)
    int n_st;                // K stages of the tensor-core path: one per site block (= nblk)
    int kind;                // INST_BLOCKS, INST_TRIPLETS or INST_DOUBLETS
    int n_fields;            // distinct input fields: 1, 3 (triplets) or 2 (doublets)
    int Nc;                  // vectors of the column field (N, except doublets of two vector counts)
    int n_sc;                // tensor-core path: site blocks of the FP64 reduction (partials per output)
    int sc_stages;           // K stages (8-site blocks) per site block of the FP64 reduction
    int out_c64;             // tensor-core path: outputs are complex64, the FP64 sums rounded once
    long long n_outB;        // output entries per timeslice: B (P C(N,3), or P N^3 for triplets; 0 if skipped)
    long long n_outM;        //                               M (P N Nc; 0 if skipped)
};

// Site-blocked layout of the tensor-core path.  phi_blk[t][b][n][TC_SLOT]:
// entry 3*o + c of slot (b, n) is 2^s phi_n^c(x = TC_BS*b + o) (zero past V),
// the last two entries are padding.  All vectors of one block are contiguous,
// so the rows' (or columns') vectors of a tile arrive with one bulk copy.
constexpr int TC_BS = 8;                      // sites per block
constexpr int TC_SLOT = 3 * TC_BS + 2;        // complex entries per (block, vector): 208 bytes

// One unit of work: a (row tile, column tile) of one timeslice -- on the
// tensor-core path restricted to one block of sites, stages [s0, s0 + nst).
// v_lo and nv give the contiguous range of vector indices the tile's rows use
// (the tensor-core path stages exactly these vectors in shared memory; for
// triplets these are phi_u vectors, and [w_lo, w_lo + nw) of phi_v follow
// them); psi_off is the byte offset of the column tile's B operand stage 0
// in the Psi buffer; part_off is the float2 offset of the tile's site block
// in the chunk's buffer of FP32 partial sums, laid out per (instance,
// timeslice) as [site block][n_outB + n_outM] in the output order.
struct TileDev {
    int inst, t, row0, col0;
    int v_lo, nv;        // vectors used by the rows: [v_lo, v_lo + nv)
    int w_lo, nw;        // triplets: phi_v vectors used by the rows (nw = 0 otherwise)
    int k_lo, nk;        // vectors used by the columns: [k_lo, k_lo + nk)
    int ncols;           // valid columns of the tile
    int cskip;           // leading columns no row of the tile needs (multiple of 8; tensor-core path)
    long long psi_off;
    int s0, nst;         // tensor-core path: first stage and number of stages of the tile's site block
    long long part_off;
};

// One (instance, timeslice) of a chunk of the tensor-core path: its Psi
// operand occupies n_ct * n_st stage images from byte psi_off of the chunk's
// Psi buffer; job0 is the index of its first (column tile, stage group) job
// within the chunk.  Its FP32 partial sums occupy n_sc * (n_outB + n_outM)
// float2 from part_off of the chunk's partial buffer; red0 is the index of
// its first block of the FP64 reduction within the chunk.
struct PsiUnit {
    int inst, t;
    long long psi_off;
    long long job0;
    long long part_off;
    long long red0;
};

__host__ __device__ inline long long binom2(long long n) { return n * (n - 1) / 2; }
__host__ __device__ inline long long binom3(long long n) { return n * (n - 1) * (n - 2) / 6; }

// Pair index q = C(j,2) + i  ->  (i, j), i < j.
__host__ __device__ inline void pair_of(long long q, int &i, int &j)
{
#ifdef __CUDA_ARCH__
    int jj = (int)((1.0 + sqrt(1.0 + 8.0 * (double)q)) * 0.5);
#else
    int jj = (int)((1.0 + __builtin_sqrt(1.0 + 8.0 * (double)q)) * 0.5);
#endif
    while (binom2(jj) > q) --jj;
    while (binom2(jj + 1) <= q) ++jj;
    j = jj;
    i = (int)(q - binom2(jj));
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// Component c of the colour cross product u x v: u^{c+1} v^{c+2} - u^{c+2} v^{c+1}
// (this is eps_cab u^a v^b).
__device__ __forceinline__ float2 cross_c(const float2 *u, const float2 *v, int c)
{
    const int a = (c + 1) % 3, b = (c + 2) % 3;
    float2 t1 = cmulf(u[a], v[b]);
    float2 t2 = cmulf(u[b], v[a]);
    return make_float2(t1.x - t2.x, t1.y - t2.y);
}

// ---- host-side launchers (defined in the .cu files) ----------------------

// laph_capi.cu: records a CUDA error for laph_last_cuda_error, returns LAPH_ERR_CUDA
int record_cuda_error(cudaError_t e, const char *where);

// laph_prep.cu
cudaError_t launch_phase_table(int L, const int32_t *d_mom, int P, double2 *out64, float2 *out32,
                               cudaStream_t s);
// fields: null (every instance has one field, phi[n]), else n_fields entries
// per instance in the order (phi, psi, chi) for triplets, (phi, psi) for
// doublets; phi may then be null.
cudaError_t launch_set_pointers(InstDev *d_inst, int first, int count, const void *const *phi,
                                void *const *outB, void *const *outM, void *workspace, cudaStream_t s,
                                const void *const *fields = nullptr, int n_fields = 1);
// Power-of-two exponent s with max|phi| * 2^s in [0.5, 1), from the FP32 bits of max|phi|.
__host__ __device__ inline int scale_exp(unsigned maxbits)
{
    if (maxbits == 0) return 0;
    int E = (int)((maxbits >> 23) & 0xff);
    if (E == 0) E = 1;
    int s = 126 - E;
    return s > 100 ? 100 : (s < -100 ? -100 : s);
}
// Max |field entry| per timeslice over all of an instance's fields (h_nfields[n] of them).
cudaError_t launch_scale_max(const InstDev *d_inst, int n_inst, const int *h_ts_base, const int *h_T,
                             const long long *h_elems, unsigned *d_maxbits, cudaStream_t s,
                             const int *h_nfields = nullptr);
cudaError_t launch_diquarks(const float2 *phi, int L, int T, int N, float2 *out, cudaStream_t s);
// Seeded pseudo-random complex entries in [-1, 1) (inputs the library makes itself).
cudaError_t launch_fill_pattern(float2 *out, long long n, unsigned seed, cudaStream_t s);
// acc[0] += sum |a - b|^2, acc[1] += sum |b|^2 (FP64; acc zeroed by the caller).
cudaError_t launch_diff_norms(const void *a, bool a_c64, const double2 *b, long long n, double *acc, cudaStream_t s);
cudaError_t launch_dense_fill(const double2 *packed, int T, int N, int P, double2 *dense, cudaStream_t s);
// Site-blocked copies of phi_u (and, for triplets, phi_v).
cudaError_t launch_blockify(const InstDev *d_inst, int inst, const InstDev &h, const unsigned *d_maxbits,
                            cudaStream_t s);
// The same for the timeslices [t0, t0 + nt) of one instance.
cudaError_t launch_scale_max_range(const InstDev *d_inst, int inst, int t0, int nt, long long elems_per_ts,
                                   unsigned *d_maxbits, cudaStream_t s, int n_fields = 1);
cudaError_t launch_blockify_range(const InstDev *d_inst, int inst, const InstDev &h, int t0, int nt,
                                  const unsigned *d_maxbits, cudaStream_t s);

// laph_simt.cu
struct SimtConfig {
    int chunk_sites;   // sites summed in FP32 before the FP64 reduction
};
constexpr int SIMT_TR = 64;  // tile rows
constexpr int SIMT_TC = 64;  // tile columns (complex)
cudaError_t launch_simt(const InstDev *d_inst, const TileDev *d_tiles, long long n_tiles,
                        const SimtConfig &cfg, int *d_status, cudaStream_t s);

// laph_tc.cu
struct TcConfig {
    int elem;          // 0 = FP16 hi/lo, 1 = BF16 hi/lo
    int ncols;         // tile width in complex columns: 104, 96, 80 or 64; row-doubled layout 208, 192, 176 or 128
    int rows2;         // 1: row-doubled layout (two real A rows per complex row, 64 complex rows per tile)
    int terms;         // 3 (split) or 1 (plain)
    int chunk_sites;   // sites accumulated by the tensor core between FP32 drains
    int chunk_sites_b; // the same for tiles without meson rows
    int grid;          // persistent CTAs
    int max_staged;    // largest number of staged row vectors (nv) of any tile
    int debug_stall;   // test hook
};
constexpr int TC_TR = 128;   // tile rows (UMMA M)
constexpr int TC_TC = 104;   // default tile columns (complex), UMMA N = 2 * TC_TC real (the widest that fits)
constexpr int TC_KSTAGE = 3 * TC_BS;  // complex K entries per stage: one site block
// One B stage image of a tile of nc complex columns: hi + lo, 2 nc real rows
// (nc in the row-doubled layout) x 48 FP16 each.
constexpr int tc_stage_bytes(int nc, bool rows2 = false) { return 2 * (rows2 ? nc : 2 * nc) * (2 * TC_KSTAGE) * 2; }
constexpr int TC_TR_ROWS2 = 64;   // complex rows per tile in the row-doubled layout
// Tile widths with compiled kernels for each layout.
bool tc_shape_supported(int ncols, int rows2);
constexpr int TC_MAX_STAGED = 160;  // staged row vectors per tile
constexpr int TC_PSI_GROUP = 16;    // stages per job of the B-operand pass
// Psi stage images of a chunk: jobs [0, n_jobs) over the units [0, n_units).
cudaError_t launch_psi(const InstDev *d_inst, const PsiUnit *d_units, int n_units, long long n_jobs,
                       const unsigned *d_maxbits, int elem, int ncols, int rows2, uint8_t *psi, cudaStream_t s);
// counter: a zeroed word of device memory; persistent CTAs claim tiles with it.
cudaError_t launch_tc(const InstDev *d_inst, const TileDev *d_tiles, long long n_tiles,
                      const unsigned *d_maxbits, const uint8_t *psi, float2 *part, unsigned *counter,
                      const TcConfig &cfg, int *d_status, cudaStream_t s);
// Output entries handled by one block of the FP64 reduction.
constexpr int TC_RED_BLOCK = 1024;
// FP64 reduction of a chunk: every output entry of the units [0, n_units) is
// the sum over its site blocks, in block order, of the FP32 partials, scaled
// back and stored to the caller's complex128 outputs.
cudaError_t launch_reduce(const InstDev *d_inst, const PsiUnit *d_units, int n_units, long long n_blocks,
                          const unsigned *d_maxbits, const float2 *part, cudaStream_t s);
// Stages in the contraction's shared-memory ring for tiles staging up to
// max_staged row vectors (0: none fits).
int tc_ring_depth(int max_staged, int ncols, int rows2);

}  // namespace laph
