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
    const void *phi[PTR_BATCH];    // column field
    const void *phi_u[PTR_BATCH];  // first row field
    const void *phi_v[PTR_BATCH];  // second row field
    void *outB[PTR_BATCH];
    void *outM[PTR_BATCH];
};

__global__ void set_pointers_kernel(InstDev *d_inst, PtrBatch b)
{
    const int n = threadIdx.x;
    if (n < b.count) {
        InstDev &I = d_inst[b.first + n];
        I.phi = (const float2 *)b.phi[n];
        I.phi_u = (const float2 *)b.phi_u[n];
        I.phi_v = (const float2 *)b.phi_v[n];
        I.outB = (double2 *)b.outB[n];
        I.outM = (double2 *)b.outM[n];
        I.phi_blk = (I.blk_off >= 0 && b.ws) ? (float2 *)(b.ws + I.blk_off) : nullptr;
        I.blk_v = (I.blkv_off >= 0 && b.ws) ? (float2 *)(b.ws + I.blkv_off) : I.phi_blk;
    }
}

cudaError_t launch_set_pointers(InstDev *d_inst, int first, int count, const void *const *phi, void *const *outB,
                                void *const *outM, void *workspace, cudaStream_t s, const void *const *fields,
                                int n_fields)
{
    for (int base = 0; base < count; base += PTR_BATCH) {
        PtrBatch b;
        b.ws = (char *)workspace;
        b.first = first + base;
        b.count = count - base < PTR_BATCH ? count - base : PTR_BATCH;
        for (int n = 0; n < b.count; n++) {
            if (!fields) {
                b.phi[n] = b.phi_u[n] = b.phi_v[n] = phi[base + n];
            } else if (n_fields == 3) {   // triplets: rows phi x psi, columns chi
                b.phi_u[n] = fields[3 * (base + n)];
                b.phi_v[n] = fields[3 * (base + n) + 1];
                b.phi[n] = fields[3 * (base + n) + 2];
            } else {                      // doublets: rows conj(phi), columns psi
                b.phi_u[n] = b.phi_v[n] = fields[2 * (base + n)];
                b.phi[n] = fields[2 * (base + n) + 1];
            }
            b.outB[n] = outB ? outB[base + n] : nullptr;
            b.outM[n] = outM ? outM[base + n] : nullptr;
        }
        set_pointers_kernel<<<1, PTR_BATCH, 0, s>>>(d_inst, b);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------- synthetic
// Seeded pseudo-random complex entries in [-1, 1) (a 32-bit integer hash of
// the index and seed), for inputs that the library makes itself (autotuning).
__global__ void fill_pattern_kernel(float2 *__restrict__ out, long long n, unsigned seed)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        unsigned h = (unsigned)i * 2654435761u ^ (unsigned)(i >> 32) * 40503u ^ seed * 2246822519u;
        h ^= h >> 15;
        h *= 2246822519u;
        h ^= h >> 13;
        h *= 3266489917u;
        h ^= h >> 16;
        const float a = (float)(h & 0xffffu) * (1.f / 32768.f) - 1.f, b = (float)(h >> 16) * (1.f / 32768.f) - 1.f;
        out[i] = make_float2(a, b);
    }
}

cudaError_t launch_fill_pattern(float2 *out, long long n, unsigned seed, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    fill_pattern_kernel<<<(unsigned)blocks, 256, 0, s>>>(out, n, seed);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- difference norms
// acc[0] += sum |a - b|^2, acc[1] += sum |b|^2 over n complex entries, a
// complex128 or complex64 (A), b complex128 (the autotuner's accuracy probe of
// a candidate schedule against the FP32 path; FP64 sums, one atomic pair per
// block).
template <typename A>
__global__ void diff_norms_kernel(const A *__restrict__ a, const double2 *__restrict__ b, long long n, double *acc)
{
    __shared__ double sd[8], sb[8];
    double d2 = 0.0, b2 = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const A xa = a[i];
        const double2 x = make_double2((double)xa.x, (double)xa.y), y = b[i];
        const double dr = x.x - y.x, di = x.y - y.y;
        d2 += dr * dr + di * di;
        b2 += y.x * y.x + y.y * y.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        d2 += __shfl_xor_sync(0xffffffffu, d2, o);
        b2 += __shfl_xor_sync(0xffffffffu, b2, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sd[w] = d2;
        sb[w] = b2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); k++) {
            d2 += sd[k];
            b2 += sb[k];
        }
        atomicAdd(acc, d2);
        atomicAdd(acc + 1, b2);
    }
}

cudaError_t launch_diff_norms(const void *a, bool a_c64, const double2 *b, long long n, double *acc, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (a_c64)
        diff_norms_kernel<float2><<<(unsigned)blocks, 256, 0, s>>>((const float2 *)a, b, n, acc);
    else
        diff_norms_kernel<double2><<<(unsigned)blocks, 256, 0, s>>>((const double2 *)a, b, n, acc);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- scale
// Largest |re|, |im| of phi per timeslice, as FP32 bits (non-negative floats
// order like their bit patterns).  The tensor-core kernel turns it into an
// exact power-of-two rescale before splitting into hi/lo halves.
__global__ void scale_max_kernel(const InstDev *__restrict__ d_inst, int inst, int t0, unsigned *__restrict__ maxbits)
{
    const InstDev &I = d_inst[inst];
    const int t = t0 + blockIdx.y;
    // field blockIdx.z: the column field (Nc vectors), then the row fields (N) of a multi-field instance
    const long long n = (long long)(blockIdx.z == 0 ? I.Nc : I.N) * I.V * 3;
    const float2 *f = blockIdx.z == 0 ? I.phi : (blockIdx.z == 1 ? I.phi_u : I.phi_v);
    const float2 *base = f + (long long)t * n;
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
                             const long long *h_elems, unsigned *d_maxbits, cudaStream_t s, const int *h_nfields)
{
    (void)h_ts_base;
    for (int n = 0; n < n_inst; n++) {
        long long blocks = (h_elems[n] + 256 * 8 - 1) / (256 * 8);
        if (blocks > 256) blocks = 256;
        if (blocks < 1) blocks = 1;
        dim3 g((unsigned)blocks, (unsigned)h_T[n], (unsigned)(h_nfields ? h_nfields[n] : 1));
        scale_max_kernel<<<g, 256, 0, s>>>(d_inst, n, 0, d_maxbits);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_scale_max_range(const InstDev *d_inst, int inst, int t0, int nt, long long elems_per_ts,
                                   unsigned *d_maxbits, cudaStream_t s, int n_fields)
{
    long long blocks = (elems_per_ts + 256 * 8 - 1) / (256 * 8);
    if (blocks > 256) blocks = 256;
    if (blocks < 1) blocks = 1;
    dim3 g((unsigned)blocks, (unsigned)nt, (unsigned)n_fields);
    scale_max_kernel<<<g, 256, 0, s>>>(d_inst, inst, t0, d_maxbits);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- site blocks
// Scaled, site-blocked copy of a row field for the tensor-core path:
// blk[t][b][n][e] = 2^s_t f[t][n][8b + e/3][e%3] for e < 24 (zero past V),
// e = 24, 25 padding, with (f, blk) = (phi_u, phi_blk) for blockIdx.z = 0 and
// (phi_v, blk_v) for blockIdx.z = 1 (triplets).  Memory bound: one read of
// the field, one write of the copy.  Block (b, t) writes the N slots of site
// block b (contiguous) and reads the 24 complex entries of each vector for
// those sites (contiguous too).
__global__ void __launch_bounds__(256) blockify_kernel(const InstDev *__restrict__ d_inst, int inst, int t0,
                                                       const unsigned *__restrict__ maxbits)
{
    const InstDev &I = d_inst[inst];
    const int b = blockIdx.x, t = t0 + blockIdx.y, N = I.N;
    const long long V = I.V;
    const float sc = __int_as_float((127 + scale_exp(maxbits[I.ts_base + t])) << 23);
    const float2 *src = (blockIdx.z ? I.phi_v : I.phi_u) + (long long)t * N * V * 3 + (long long)TC_BS * b * 3;
    float2 *dst = (blockIdx.z ? I.blk_v : I.phi_blk) + ((long long)t * I.nblk + b) * N * TC_SLOT;
    const int nvalid = (int)(V - (long long)TC_BS * b < TC_BS ? V - (long long)TC_BS * b : TC_BS) * 3;
    for (int idx = threadIdx.x; idx < N * TC_SLOT; idx += blockDim.x) {
        const int n = idx / TC_SLOT, e = idx - n * TC_SLOT;
        float2 v = make_float2(0.f, 0.f);
        if (e < nvalid) {
            const float2 f = __ldg(src + (long long)n * V * 3 + e);
            v = make_float2(f.x * sc, f.y * sc);
        }
        dst[idx] = v;
    }
}

cudaError_t launch_blockify(const InstDev *d_inst, int inst, const InstDev &h, const unsigned *d_maxbits, cudaStream_t s)
{
    return launch_blockify_range(d_inst, inst, h, 0, h.T, d_maxbits, s);
}

cudaError_t launch_blockify_range(const InstDev *d_inst, int inst, const InstDev &h, int t0, int nt,
                                  const unsigned *d_maxbits, cudaStream_t s)
{
    for (int tb = 0; tb < nt; tb += 65535) {
        const int n = nt - tb < 65535 ? nt - tb : 65535;
        dim3 g((unsigned)h.nblk, (unsigned)n, h.kind == INST_TRIPLETS ? 2u : 1u);
        blockify_kernel<<<g, 256, 0, s>>>(d_inst, inst, t0 + tb, d_maxbits);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------- K-b
// D[t][q][x][c] = (phi_i(x) x phi_j(x))_c for q = C(j,2) + i.  One block per
// (block of DQ_SB = 64 sites, timeslice): phi of all N vectors for those
// sites is staged in shared memory, then every warp takes one pair at a time
// and each lane forms two whole sites (6 complex, three 16-byte loads per
// vector, 48 FMAs).  The lane's 48 bytes go through a per-warp shared buffer
// so that each global store instruction writes 512 contiguous bytes.
constexpr int DQ_SB = 64;
constexpr int DQ_THREADS = 256;

__global__ void __launch_bounds__(DQ_THREADS) diquark_kernel(const float2 *__restrict__ phi, int N, long long V,
                                                             float2 *__restrict__ out)
{
    extern __shared__ float4 dq_smem[];
    float2 *sphi = reinterpret_cast<float2 *>(dq_smem);          // [N][DQ_SB][3]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = DQ_THREADS / 32;
    float4 *xbuf = dq_smem + (size_t)N * DQ_SB * 3 / 2 + warp * 96; // per warp: 96 x 16 bytes
    const int t = blockIdx.y;
    const long long x0 = (long long)blockIdx.x * DQ_SB;
    const int nsite = (int)((V - x0) < DQ_SB ? (V - x0) : DQ_SB);
    const bool aligned = (V & 1) == 0;   // 16-byte aligned rows of phi and D
    const float2 *src = phi + (long long)t * N * V * 3;
    const int w3 = DQ_SB * 3;
    // stage phi[t][n][x0 .. x0+nsite)[3], zero past V
    if (aligned) {
        const int q4 = w3 / 2;   // float4 per vector
        for (int idx = threadIdx.x; idx < N * q4; idx += DQ_THREADS) {
            const int n = idx / q4, e = idx - n * q4;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (2 * e < nsite * 3) v = __ldg(reinterpret_cast<const float4 *>(src + ((long long)n * V + x0) * 3) + e);
            dq_smem[idx] = v;
        }
    } else {
        for (int idx = threadIdx.x; idx < N * w3; idx += DQ_THREADS) {
            const int n = idx / w3, e = idx - n * w3;
            sphi[idx] = e < nsite * 3 ? __ldg(src + ((long long)n * V + x0) * 3 + e) : make_float2(0.f, 0.f);
        }
    }
    __syncthreads();
    const long long pairs = binom2(N);
    int i = 0, j = 1;
    if (warp < pairs) pair_of(warp, i, j);
    for (long long q = warp; q < pairs; q += nwarp) {
        // sites 2 lane, 2 lane + 1 of vectors i and j
        const float4 *u4 = reinterpret_cast<const float4 *>(sphi + ((long long)i * DQ_SB + 2 * lane) * 3);
        const float4 *v4 = reinterpret_cast<const float4 *>(sphi + ((long long)j * DQ_SB + 2 * lane) * 3);
        float2 u[6], v[6];
#pragma unroll
        for (int h = 0; h < 3; h++) {
            const float4 a = u4[h], b = v4[h];
            u[2 * h] = make_float2(a.x, a.y);
            u[2 * h + 1] = make_float2(a.z, a.w);
            v[2 * h] = make_float2(b.x, b.y);
            v[2 * h + 1] = make_float2(b.z, b.w);
        }
        float2 d[6];
#pragma unroll
        for (int e = 0; e < 6; e++) d[e] = cross_c(u + 3 * (e / 3), v + 3 * (e / 3), e % 3);
        float2 *dst = out + (((long long)t * pairs + q) * V + x0) * 3;
        if (aligned && nsite == DQ_SB) {
            // transpose through the warp's buffer: lane l holds float4 3l..3l+2 of the pair's 96
#pragma unroll
            for (int h = 0; h < 3; h++) xbuf[3 * lane + h] = make_float4(d[2 * h].x, d[2 * h].y, d[2 * h + 1].x, d[2 * h + 1].y);
            __syncwarp();
#pragma unroll
            for (int h = 0; h < 3; h++) reinterpret_cast<float4 *>(dst)[32 * h + lane] = xbuf[32 * h + lane];
            __syncwarp();
        } else {
#pragma unroll
            for (int e = 0; e < 6; e++)
                if (6 * lane + e < nsite * 3) dst[6 * lane + e] = d[e];
        }
        // next pair of this warp: q + nwarp
        const long long qn = q + nwarp;
        if (qn < pairs) {
            i += nwarp;
            while (i >= j) {
                i -= j;
                j++;
            }
        }
    }
}

// Vector counts whose staged sites do not fit in shared memory: one thread per
// output entry, operands read from global memory.
__global__ void diquark_generic_kernel(const float2 *__restrict__ phi, int N, long long V, long long total,
                                       float2 *__restrict__ out)
{
    const long long pairs = binom2(N);
    for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < total; o += (long long)gridDim.x * blockDim.x) {
        const long long e = o % (3 * V), r = o / (3 * V);
        const long long q = r % pairs, t = r / pairs;
        int i, j;
        pair_of(q, i, j);
        const long long x = e / 3;
        const int c = (int)(e - 3 * x);
        const float2 *u = phi + ((t * N + i) * V + x) * 3, *v = phi + ((t * N + j) * V + x) * 3;
        float2 uu[3] = {__ldg(u), __ldg(u + 1), __ldg(u + 2)}, vv[3] = {__ldg(v), __ldg(v + 1), __ldg(v + 2)};
        out[o] = cross_c(uu, vv, c);
    }
}

cudaError_t launch_diquarks(const float2 *phi, int L, int T, int N, float2 *out, cudaStream_t s)
{
    const long long V = (long long)L * L * L;
    const size_t smem = (size_t)N * DQ_SB * 3 * sizeof(float2) + (DQ_THREADS / 32) * 96 * 16;
    if (smem > 227 * 1024) {
        const long long total = (long long)T * binom2(N) * 3 * V;
        long long blocks = (total + 255) / 256;
        if (blocks > 152 * 64) blocks = 152 * 64;
        diquark_generic_kernel<<<(unsigned)blocks, 256, 0, s>>>(phi, N, V, total, out);
        return cudaGetLastError();
    }
    cudaError_t e = cudaFuncSetAttribute(diquark_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 g((unsigned)((V + DQ_SB - 1) / DQ_SB), (unsigned)T);
    diquark_kernel<<<g, DQ_THREADS, smem, s>>>(phi, N, V, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- K-g
// dense[t][p][a][b][c] = sign * packed[t][p][C(k,3)+C(j,2)+i] with (i,j,k) the
// sorted (a,b,c) and sign the parity of the sort (the product of the signs
// of b-a, c-a and c-b); 0 on a repeated index.  Block (a, tp) writes the N*N
// entries (b, c) of row a, c fastest; no branches depend on the indices.
__global__ void __launch_bounds__(256) dense_fill_kernel(const double2 *__restrict__ packed, int N, long long n_trip,
                                                         long long tp0, double2 *__restrict__ dense)
{
    const int a = blockIdx.x;
    const long long tp = tp0 + blockIdx.y;
    const double2 *pk = packed + tp * n_trip;
    double2 *row = dense + (tp * N + a) * (long long)N * N;
    const int nn = N * N;
    // eight gathers per thread are issued before their stores, so that enough
    // of the (L2-resident) packed loads are in flight to keep the writes streaming
    constexpr int BATCH = 8;
    for (int r0 = 0; r0 < nn; r0 += 256 * BATCH) {
        double2 w[BATCH];
        bool neg[BATCH];
#pragma unroll
        for (int q = 0; q < BATCH; q++) {
            const int r = r0 + q * 256 + threadIdx.x;
            w[q] = make_double2(0.0, 0.0);
            neg[q] = false;
            if (r < nn) {
                const int b = r / N, c = r - b * N;
                const int lo = min(a, min(b, c)), hi = max(a, max(b, c)), mid = a + b + c - lo - hi;
                const bool rep = (a == b) | (b == c) | (a == c);
                neg[q] = !rep && ((b < a) ^ (c < a) ^ (c < b));   // repeated indices give +0
                if (!rep) w[q] = __ldg(pk + binom3(hi) + binom2(mid) + lo);
            }
        }
#pragma unroll
        for (int q = 0; q < BATCH; q++) {
            const int r = r0 + q * 256 + threadIdx.x;
            if (r < nn) row[r] = neg[q] ? make_double2(-w[q].x, -w[q].y) : w[q];
        }
    }
}

cudaError_t launch_dense_fill(const double2 *packed, int T, int N, int P, double2 *dense, cudaStream_t s)
{
    const long long TP = (long long)T * P;
    for (long long tp0 = 0; tp0 < TP; tp0 += 65535) {
        const long long n = TP - tp0 < 65535 ? TP - tp0 : 65535;
        dim3 g((unsigned)N, (unsigned)n);
        dense_fill_kernel<<<g, 256, 0, s>>>(packed, N, binom3(N), tp0, dense);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace laph
