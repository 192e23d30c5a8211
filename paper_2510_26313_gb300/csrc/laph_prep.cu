// Small kernels around the contraction: the momentum phase table (K-a), the
// pointer upload for a batch, the per-timeslice power-of-two scale used by
// the tensor-core split, the materialised diquark stage (K-b) and the dense
// antisymmetric fill of the packed baryon blocks (K-g).
#include "laph_internal.cuh"

namespace laph {

// ---------------------------------------------------------------- K-a
// ph_p(x) = exp(-2 pi i r / L), r = (n_p . x) mod L in [0, L), evaluated in
// FP64 with sincospi on the exactly reduced integer argument (momentum
// projection of section "Innovations"/"QUDA").
__global__ void phase_table_kernel(int L, const int32_t *__restrict__ mom, int P, long long V, long long Vs,
                                   double2 *__restrict__ out64, float2 *__restrict__ out32)
{
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)P * V) return;
    const int p = (int)(idx / V);
    const long long x = idx - (long long)p * V;
    const long long x0 = x % L, x1 = (x / L) % L, x2 = x / ((long long)L * L);
    long long r = ((long long)mom[3 * p] * x0 + (long long)mom[3 * p + 1] * x1 + (long long)mom[3 * p + 2] * x2) % L;
    if (r < 0) r += L;
    double s, c;
    sincospi(-2.0 * (double)r / (double)L, &s, &c);
    if (out64) out64[idx] = make_double2(c, s);
    if (out32) out32[p * Vs + x] = make_float2((float)c, (float)s);
}

cudaError_t launch_phase_table(int L, const int32_t *d_mom, int P, double2 *out64, float2 *out32, cudaStream_t s)
{
    const long long V = (long long)L * L * L;
    const long long Vs = V + (V & 1);
    const long long n = (long long)P * V;
    const int bs = 256;
    const long long nb = (n + bs - 1) / bs;
    phase_table_kernel<<<(unsigned)nb, bs, 0, s>>>(L, d_mom, P, V, Vs, out64, out32);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- pointers
// The caller's buffer pointers reach the device through kernel parameters,
// which a stream capture records by value: no host memory is read later.
constexpr int PTR_BATCH = 64;
struct PtrBatch {
    int first, count;
    char *ws;
    const void *phi[PTR_BATCH];
    void *outB[PTR_BATCH];
    void *outM[PTR_BATCH];
};

__global__ void set_pointers_kernel(InstDev *d_inst, PtrBatch b)
{
    const int n = threadIdx.x;
    if (n < b.count) {
        InstDev &I = d_inst[b.first + n];
        I.phi = (const float2 *)b.phi[n];
        I.outB = (double2 *)b.outB[n];
        I.outM = (double2 *)b.outM[n];
        I.phi_blk = (I.blk_off >= 0 && b.ws) ? (float2 *)(b.ws + I.blk_off) : nullptr;
    }
}

cudaError_t launch_set_pointers(InstDev *d_inst, int first, int count, const void *const *phi, void *const *outB,
                                void *const *outM, void *workspace, cudaStream_t s)
{
    for (int base = 0; base < count; base += PTR_BATCH) {
        PtrBatch b;
        b.ws = (char *)workspace;
        b.first = first + base;
        b.count = count - base < PTR_BATCH ? count - base : PTR_BATCH;
        for (int n = 0; n < b.count; n++) {
            b.phi[n] = phi[base + n];
            b.outB[n] = outB ? outB[base + n] : nullptr;
            b.outM[n] = outM ? outM[base + n] : nullptr;
        }
        set_pointers_kernel<<<1, PTR_BATCH, 0, s>>>(d_inst, b);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------- scale
// Largest |re|, |im| of phi per timeslice, as FP32 bits (non-negative floats
// order like their bit patterns).  The tensor-core kernel turns it into an
// exact power-of-two rescale before splitting into hi/lo halves.
__global__ void scale_max_kernel(const InstDev *__restrict__ d_inst, int inst, unsigned *__restrict__ maxbits)
{
    const InstDev &I = d_inst[inst];
    const int t = blockIdx.y;
    const long long n = (long long)I.N * I.V * 3;
    const float2 *base = I.phi + (long long)t * n;
    float m = 0.f;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        float2 v = __ldg(base + e);
        m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) atomicMax(maxbits + I.ts_base + t, __float_as_uint(m));
    }
}

cudaError_t launch_scale_max(const InstDev *d_inst, int n_inst, const int *h_ts_base, const int *h_T,
                             const long long *h_elems, unsigned *d_maxbits, cudaStream_t s)
{
    (void)h_ts_base;
    for (int n = 0; n < n_inst; n++) {
        long long blocks = (h_elems[n] + 256 * 8 - 1) / (256 * 8);
        if (blocks > 256) blocks = 256;
        if (blocks < 1) blocks = 1;
        dim3 g((unsigned)blocks, (unsigned)h_T[n]);
        scale_max_kernel<<<g, 256, 0, s>>>(d_inst, n, d_maxbits);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------- site blocks
// Scaled, site-blocked copy of phi for the tensor-core path:
// phi_blk[t][b][n][e] = 2^s_t phi[t][n][8b + e/3][e%3] for e < 24 (zero past V),
// e = 24, 25 padding.  Memory bound: one read of phi, one write of the copy.
__global__ void blockify_kernel(const InstDev *__restrict__ d_inst, int inst, const unsigned *__restrict__ maxbits)
{
    const InstDev &I = d_inst[inst];
    const long long total = (long long)I.T * I.nblk * I.N * TC_SLOT;
    const long long V = I.V;
    for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < total; o += (long long)gridDim.x * blockDim.x) {
        const long long chunk = o / TC_SLOT;
        const int e = (int)(o - chunk * TC_SLOT);
        const int n = (int)(chunk % I.N);
        const long long tb = chunk / I.N;
        const int b = (int)(tb % I.nblk);
        const int t = (int)(tb / I.nblk);
        const long long x = (long long)TC_BS * b + e / 3;
        float2 v = make_float2(0.f, 0.f);
        if (e < 3 * TC_BS && x < V) {
            const float sc = __int_as_float((127 + scale_exp(maxbits[I.ts_base + t])) << 23);
            const float2 f = __ldg(I.phi + (((long long)t * I.N + n) * V + x) * 3 + e % 3);
            v = make_float2(f.x * sc, f.y * sc);
        }
        I.phi_blk[o] = v;
    }
}

cudaError_t launch_blockify(const InstDev *d_inst, int inst, const InstDev &h, const unsigned *d_maxbits, cudaStream_t s)
{
    const long long n = (long long)h.T * h.nblk * h.N * TC_SLOT;
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    blockify_kernel<<<(unsigned)blocks, 256, 0, s>>>(d_inst, inst, d_maxbits);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- K-b
// D[t][q][x][c] = (phi_i(x) x phi_j(x))_c for q = C(j,2) + i.  One block per
// (site block of SB sites, timeslice): phi of all N vectors for those sites
// is staged in shared memory with 16-byte loads, then every warp writes whole
// pairs, SB*3 complex numbers per pair, as contiguous 16-byte stores.
__global__ void diquark_kernel(const float2 *__restrict__ phi, int N, long long V, int SB, float2 *__restrict__ out)
{
    extern __shared__ float2 sphi[];  // [N][SB*3]
    const int t = blockIdx.y;
    const long long x0 = (long long)blockIdx.x * SB;
    const int nsite = (int)((V - x0) < SB ? (V - x0) : SB);
    const int w3 = SB * 3;
    const float2 *src = phi + (long long)t * N * V * 3;
    // stage: vector n, complex e in [0, nsite*3)
    for (int idx = threadIdx.x; idx < N * w3; idx += blockDim.x) {
        const int n = idx / w3, e = idx - n * w3;
        sphi[idx] = e < nsite * 3 ? __ldg(src + ((long long)n * V + x0) * 3 + e) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const long long pairs = binom2(N);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    const bool vec4 = ((V & 1) == 0) && (nsite == SB);  // 16-byte aligned whole rows
    for (long long q = warp; q < pairs; q += nwarp) {
        int i, j;
        pair_of(q, i, j);
        const float2 *u = sphi + i * w3, *v = sphi + j * w3;
        float2 *dst = out + (((long long)t * pairs + q) * V + x0) * 3;
        if (vec4) {
            for (int f = lane; f < w3 / 2; f += 32) {
                float2 r[2];
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const int e = 2 * f + h, x = e / 3, c = e - 3 * x;
                    r[h] = cross_c(u + 3 * x, v + 3 * x, c);
                }
                reinterpret_cast<float4 *>(dst)[f] = make_float4(r[0].x, r[0].y, r[1].x, r[1].y);
            }
        } else {
            for (int e = lane; e < nsite * 3; e += 32) {
                const int x = e / 3, c = e - 3 * x;
                dst[e] = cross_c(u + 3 * x, v + 3 * x, c);
            }
        }
    }
}

cudaError_t launch_diquarks(const float2 *phi, int L, int T, int N, float2 *out, cudaStream_t s)
{
    const long long V = (long long)L * L * L;
    int SB = 32;
    while (SB > 2 && (long long)N * SB * 3 * 8 > 160 * 1024) SB /= 2;
    const size_t smem = (size_t)N * SB * 3 * sizeof(float2);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(diquark_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 g((unsigned)((V + SB - 1) / SB), (unsigned)T);
    diquark_kernel<<<g, 256, smem, s>>>(phi, N, V, SB, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- K-g
// dense[t][p][a][b][c] = sign * packed[t][p][C(k,3)+C(j,2)+i] with (i,j,k) the
// sorted (a,b,c) and sign the parity of the sort; 0 on a repeated index.
__global__ void dense_fill_kernel(const double2 *__restrict__ packed, int N, long long n_trip, long long total,
                                  double2 *__restrict__ dense)
{
    const long long n3 = (long long)N * N * N;
    for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < total; o += (long long)gridDim.x * blockDim.x) {
        const long long tp = o / n3;
        const long long r = o - tp * n3;
        int a = (int)(r / ((long long)N * N)), b = (int)((r / N) % N), c = (int)(r % N);
        double sgn = 1.0;
        int t0;
        if (a > b) { t0 = a; a = b; b = t0; sgn = -sgn; }
        if (b > c) { t0 = b; b = c; c = t0; sgn = -sgn; }
        if (a > b) { t0 = a; a = b; b = t0; sgn = -sgn; }
        double2 v = make_double2(0.0, 0.0);
        if (a != b && b != c) {
            const double2 s = packed[tp * n_trip + binom3(c) + binom2(b) + a];
            v = make_double2(sgn * s.x, sgn * s.y);
        }
        dense[o] = v;
    }
}

cudaError_t launch_dense_fill(const double2 *packed, int T, int N, int P, double2 *dense, cudaStream_t s)
{
    const long long total = (long long)T * P * N * N * N;
    long long blocks = (total + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    if (blocks < 1) blocks = 1;
    dense_fill_kernel<<<(unsigned)blocks, 256, 0, s>>>(packed, N, binom3(N), total, dense);
    return cudaGetLastError();
}

}  // namespace laph
