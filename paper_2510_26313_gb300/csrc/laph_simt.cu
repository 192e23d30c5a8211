// FP32 CUDA-core path of the block contraction (K-h).
//
// The contraction is a complex matrix product over K = 3V (site, colour):
//   C[row][col] = sum_{x,c} A[row](x,c) * Psi[col](x,c)
// with A = conj(phi_i) for a meson row i, A = (phi_i x phi_j) (the diquark,
// eps_cab phi_i^a phi_j^b) for a pair row (i<j), and Psi[(k,p)] = ph_p(x) phi_k.
// Then M[p][i][k] = C[i][(k,p)] and B[p][i,j,k] = C[(i,j)][(k,p)] for k > j.
//
// One block computes a 64-row x 64-column tile of one timeslice; the tile
// table skips tiles that lie wholly below the k > j triangle.  Per chunk of
// 16 sites the block forms the A and Psi operands in shared memory and every
// thread accumulates a 4x4 complex micro-tile in FP32.  Every chunk_sites
// sites the FP32 partial sums are added in FP64 into the output, which each
// element's owner thread alone reads and writes (first chunk stores).
#include "laph_internal.cuh"

namespace laph {

namespace {
constexpr int KS = 16;               // sites per shared-memory chunk
constexpr int KC = 3 * KS;           // complex K entries per chunk
constexpr int APITCH = SIMT_TR + 2;  // float2 pitch, 16-byte aligned rows
constexpr int BPITCH = SIMT_TC + 2;
constexpr int NTHREADS = 256;
static_assert(SIMT_TR == 64 && SIMT_TC == 64, "thread mapping assumes 64x64 tiles");
}  // namespace

__global__ void __launch_bounds__(NTHREADS, 2)
simt_kernel(const InstDev *__restrict__ insts, const TileDev *__restrict__ tiles, int chunk_sites)
{
    extern __shared__ __align__(16) float2 sm[];
    float2 *As = sm;                 // [KC][APITCH]
    float2 *Bs = sm + KC * APITCH;   // [KC][BPITCH]

    const TileDev tile = tiles[blockIdx.x];
    const InstDev I = insts[tile.inst];
    const int tid = threadIdx.x;
    const long long V = I.V;
    const int N = I.N, P = I.P;
    const float2 *__restrict__ phit = I.phi + (long long)tile.t * N * V * 3;
    const float2 *__restrict__ ph = I.phase;

    // ---- operand-production mapping: site s, rows/cols tid/KS + 16*m
    const int s = tid % KS;
    int ai[4], aj[4], bk[4], bp[4];
#pragma unroll
    for (int m = 0; m < 4; m++) {
        const int r = tid / KS + 16 * m;
        const int g = tile.row0 + r;
        if (g >= I.rows) {
            ai[m] = -1;
            aj[m] = -1;
        } else if (g < I.mes_rows) {
            ai[m] = g;
            aj[m] = -1;
        } else {
            int i, j;
            pair_of(g - I.mes_rows, i, j);
            ai[m] = i;
            aj[m] = j;
        }
        const int col = tile.col0 + r;
        if (col >= I.cols) {
            bk[m] = -1;
            bp[m] = 0;
        } else {
            bk[m] = col / P;
            bp[m] = col - bk[m] * P;
        }
    }

    // ---- accumulation mapping: rows ty*4+m, cols tx*4+n
    const int ty = tid / 16, tx = tid % 16;
    float2 acc[4][4];
#pragma unroll
    for (int m = 0; m < 4; m++)
#pragma unroll
        for (int n = 0; n < 4; n++) acc[m][n] = make_float2(0.f, 0.f);

    const long long nchunks = (V + KS - 1) / KS;
    int since = 0;
    bool first_drain = true;

    for (long long ch = 0; ch < nchunks; ch++) {
        const long long x = ch * KS + s;
        const bool xin = x < V;
#pragma unroll
        for (int m = 0; m < 4; m++) {
            float2 o[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
            if (xin && ai[m] >= 0) {
                const float2 *u = phit + ((long long)ai[m] * V + x) * 3;
                float2 uu[3] = {__ldg(u), __ldg(u + 1), __ldg(u + 2)};
                if (aj[m] < 0) {
#pragma unroll
                    for (int c = 0; c < 3; c++) o[c] = conjf2(uu[c]);
                } else {
                    const float2 *v = phit + ((long long)aj[m] * V + x) * 3;
                    float2 vv[3] = {__ldg(v), __ldg(v + 1), __ldg(v + 2)};
#pragma unroll
                    for (int c = 0; c < 3; c++) o[c] = cross_c(uu, vv, c);
                }
            }
            const int r = tid / KS + 16 * m;
#pragma unroll
            for (int c = 0; c < 3; c++) As[(3 * s + c) * APITCH + r] = o[c];
        }
#pragma unroll
        for (int m = 0; m < 4; m++) {
            float2 o[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
            if (xin && bk[m] >= 0) {
                const float2 *w = phit + ((long long)bk[m] * V + x) * 3;
                const float2 phv = __ldg(ph + (long long)bp[m] * I.Vs + x);
#pragma unroll
                for (int c = 0; c < 3; c++) o[c] = cmulf(phv, __ldg(w + c));
            }
            const int cl = tid / KS + 16 * m;
#pragma unroll
            for (int c = 0; c < 3; c++) Bs[(3 * s + c) * BPITCH + cl] = o[c];
        }
        __syncthreads();

#pragma unroll 4
        for (int kk = 0; kk < KC; kk++) {
            const float4 a01 = *reinterpret_cast<const float4 *>(As + kk * APITCH + ty * 4);
            const float4 a23 = *reinterpret_cast<const float4 *>(As + kk * APITCH + ty * 4 + 2);
            const float4 b01 = *reinterpret_cast<const float4 *>(Bs + kk * BPITCH + tx * 4);
            const float4 b23 = *reinterpret_cast<const float4 *>(Bs + kk * BPITCH + tx * 4 + 2);
            const float2 a[4] = {make_float2(a01.x, a01.y), make_float2(a01.z, a01.w), make_float2(a23.x, a23.y),
                                 make_float2(a23.z, a23.w)};
            const float2 b[4] = {make_float2(b01.x, b01.y), make_float2(b01.z, b01.w), make_float2(b23.x, b23.y),
                                 make_float2(b23.z, b23.w)};
#pragma unroll
            for (int m = 0; m < 4; m++)
#pragma unroll
                for (int n = 0; n < 4; n++) {
                    acc[m][n].x = fmaf(a[m].x, b[n].x, acc[m][n].x);
                    acc[m][n].x = fmaf(-a[m].y, b[n].y, acc[m][n].x);
                    acc[m][n].y = fmaf(a[m].x, b[n].y, acc[m][n].y);
                    acc[m][n].y = fmaf(a[m].y, b[n].x, acc[m][n].y);
                }
        }
        __syncthreads();

        since += KS;
        if (since >= chunk_sites || ch == nchunks - 1) {
            // ---- FP64 reduction of this chunk's partial sums into the output
#pragma unroll
            for (int m = 0; m < 4; m++) {
                const int g = tile.row0 + ty * 4 + m;
                if (g >= I.rows) continue;
                const bool meson = g < I.mes_rows;
                int pi = 0, pj = 0;
                long long q = 0;
                if (!meson) {
                    q = g - I.mes_rows;
                    pair_of(q, pi, pj);
                }
#pragma unroll
                for (int n = 0; n < 4; n++) {
                    const int col = tile.col0 + tx * 4 + n;
                    if (col >= I.cols) continue;
                    const int k = col / P, p = col - k * P;
                    double2 *dst;
                    if (meson) {
                        dst = I.outM + (((long long)tile.t * P + p) * N + g) * N + k;
                    } else {
                        if (k <= pj) continue;
                        dst = I.outB + ((long long)tile.t * P + p) * I.n_trip + binom3(k) + q;
                    }
                    double2 v = make_double2((double)acc[m][n].x, (double)acc[m][n].y);
                    if (!first_drain) {
                        const double2 old = *dst;
                        v.x += old.x;
                        v.y += old.y;
                    }
                    *dst = v;
                }
            }
#pragma unroll
            for (int m = 0; m < 4; m++)
#pragma unroll
                for (int n = 0; n < 4; n++) acc[m][n] = make_float2(0.f, 0.f);
            since = 0;
            first_drain = false;
        }
    }
}

cudaError_t launch_simt(const InstDev *d_inst, const TileDev *d_tiles, long long n_tiles, const SimtConfig &cfg,
                        int *d_status, cudaStream_t s)
{
    (void)d_status;
    if (n_tiles <= 0) return cudaSuccess;
    const size_t smem = (size_t)KC * (APITCH + BPITCH) * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(simt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int chunk = cfg.chunk_sites > 0 ? cfg.chunk_sites : 1024;
    for (long long base = 0; base < n_tiles; base += 0x7fffffffLL) {
        const long long n = (n_tiles - base) < 0x7fffffffLL ? (n_tiles - base) : 0x7fffffffLL;
        simt_kernel<<<(unsigned)n, NTHREADS, smem, s>>>(d_inst, d_tiles + base, chunk);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace laph
