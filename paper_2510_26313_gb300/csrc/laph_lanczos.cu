// The 3-d gauge-covariant Laplacian of every timeslice and a batched Lanczos
// eigensolver for its lowest eigenpairs, the LapH eigenvectors (paper,
// section "Innovations", subsection "Scalable Lanczos Eigensolver": the
// timeslices are independent problems, solved side by side, with no
// communication between them).
//
//   (-Delta f)(x) = sum_mu [ 2 f(x) - U_mu(x) f(x + mu) - U_mu(x - mu)^dagger f(x - mu) ]
//
// Layouts (complex interleaved): links U [T][3][V][3][3] complex64 (row-major
// colour matrices), vectors [T][n][V][3] complex64, site x = x0 + L x1 + L^2 x2.
//
// Lanczos with full reorthogonalisation, batched over timeslices: every
// iteration applies the operator to the newest basis vector of every
// timeslice, removes its components along the whole basis twice ("twice is
// enough"), and normalises.  The operator is -Delta itself or the Chebyshev
// filter T_d((-Delta - c) / e), which maps the unwanted part of the spectrum,
// [lo, 12], onto [-1, 1] and magnifies the lowest eigenvalues.  The Ritz
// vectors of the wanted end are formed from the basis (host symmetric QR on the
// tridiagonal matrices), and their eigenvalues and residuals are Rayleigh
// quotients with -Delta.
//
// Precision: FP32 vectors and links; inner products are FP32 products summed
// in FP32 within a thread and a warp and in FP64 across warps and blocks.
// Layout and scheduling: the solver copies the links into its own
// structure-of-arrays layout (16-byte pairs where V is even) and keeps its
// vectors in the matching layout; the filter runs group by group of
// timeslices that fit in L2, all its steps replayed as one CUDA graph per
// Krylov step.
#include <algorithm>
#include <limits>
#include <cmath>
#include <cstring>
#include <initializer_list>
#include <thread>
#include <vector>

#include "laph.h"
#include "laph_internal.cuh"

namespace laph {
namespace {

constexpr int LAP_THREADS = 256;
// launch shape of the solver's stencil (tuning: block size, minimum resident
// blocks per SM, and 1 to read the links past L1)
#ifndef LAP_SOA_THREADS
#define LAP_SOA_THREADS 256
#endif
#ifndef LAP_SOA_MINB
#define LAP_SOA_MINB 4
#endif
#ifndef LAP_SOA_LINKS_CG
#define LAP_SOA_LINKS_CG 0
#endif

__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 acc)   // acc + a b
{
    return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y)));
}

__device__ __forceinline__ float2 cfma_conj(float2 a, float2 b, float2 acc)   // acc + conj(a) b
{
    return make_float2(fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x)), fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y)));
}

// out = a (-Delta in) + b in + c z for vector blockIdx.y of timeslice
// blockIdx.z (the vectors of a timeslice run together and share its links in
// L2); one thread per site.  in/z/out: [T][nvec][V][3] with the given
// per-timeslice strides (in elements of float2); z may be null (c ignored).
__global__ void __launch_bounds__(LAP_THREADS, 4) lap_kernel(const float2 *__restrict__ U, const float2 *__restrict__ in,
                                                          const float2 *__restrict__ z, float2 *__restrict__ out,
                                                          int L, long long ts_in, long long ts_z, long long ts_out,
                                                          float a, float b, float c)
{
    const long long V = (long long)L * L * L;
    const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= V) return;
    const int n = blockIdx.y, t = blockIdx.z;
    const float2 *f = in + t * ts_in + n * V * 3;
    const float2 *Ut = U + (long long)t * 3 * V * 9;
    const int c0 = (int)(x % L), c1 = (int)((x / L) % L), c2 = (int)(x / ((long long)L * L));
    const int cc[3] = {c0, c1, c2};
    const long long stride[3] = {1, L, (long long)L * L};
    float2 fx[3], acc[3];
#pragma unroll
    for (int q = 0; q < 3; q++) {
        fx[q] = f[3 * x + q];
        acc[q] = make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int mu = 0; mu < 3; mu++) {
        const long long up = x + (cc[mu] == L - 1 ? -(long long)(L - 1) * stride[mu] : stride[mu]);
        const long long dn = x - (cc[mu] == 0 ? -(long long)(L - 1) * stride[mu] : stride[mu]);
        const float2 *pf = Ut + (mu * V + x) * 9;     // U_mu(x)
        const float2 *pb = Ut + (mu * V + dn) * 9;    // U_mu(x - mu)
        // all loads of this direction issued before its multiply-adds
        float2 fu[3], fd[3], uf[9], ub[9];
#pragma unroll
        for (int q = 0; q < 3; q++) {
            fu[q] = f[3 * up + q];
            fd[q] = f[3 * dn + q];
        }
#pragma unroll
        for (int k = 0; k < 9; k++) {
            uf[k] = __ldg(pf + k);
            ub[k] = __ldg(pb + k);
        }
#pragma unroll
        for (int r = 0; r < 3; r++)
#pragma unroll
            for (int q = 0; q < 3; q++) {
                acc[r] = cfma(uf[3 * r + q], fu[q], acc[r]);          // U_mu(x)_{rq} f_q(x + mu)
                acc[r] = cfma_conj(ub[3 * q + r], fd[q], acc[r]);     // conj(U_mu(x - mu)_{qr}) f_q(x - mu)
            }
    }
    float2 *o = out + t * ts_out + n * V * 3 + 3 * x;
    const float2 *zz = z ? z + t * ts_z + n * V * 3 + 3 * x : nullptr;
#pragma unroll
    for (int q = 0; q < 3; q++) {
        // -Delta f = 6 f(x) - (hops)
        float2 lap = make_float2(6.f * fx[q].x - acc[q].x, 6.f * fx[q].y - acc[q].y);
        float2 r = make_float2(a * lap.x + b * fx[q].x, a * lap.y + b * fx[q].y);
        if (zz) {
            r.x += c * zz[q].x;
            r.y += c * zz[q].y;
        }
        o[q] = r;
    }
}

// The third row of an SU(3) matrix from its first two: row2 = conj(row0 x row1)
// (its rows are orthonormal and its determinant, row2 . (row0 x row1), is 1).
__device__ __forceinline__ void su3_third_row(float2 *u)
{
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
        const float2 a = u[k1], b = u[3 + k2], c = u[k2], e = u[3 + k1];
        // (a b - c e)^*
        const float re = a.x * b.x - a.y * b.y - (c.x * e.x - c.y * e.y);
        const float im = a.x * b.y + a.y * b.x - (c.x * e.y + c.y * e.x);
        u[6 + k] = make_float2(re, -im);
    }
}

// The solver's own layouts, in which a warp reads consecutive sites:
// - plain: links Us [T][3][9][V] (direction, row-major colour entry, site),
//   vectors [3][V] (colour, site);
// - paired (V even, so that every block is 16-byte aligned): the links of a
//   direction are entries (0,1), (2,3), (4,5), (6,7) as four [V] arrays of
//   16-byte pairs, then entry 8 as a [V] array; a vector is colours (0,1) as
//   a [V] array of pairs, then colour 2 as a [V] array.  A site's vector is two
//   loads instead of three, a link five instead of nine.
// The orthogonalisation and Ritz kernels treat a vector as 3V elements in any
// order; the final gather writes the caller's [V][3].
template <bool PAIRS>
__device__ __forceinline__ void load_site(const float2 *__restrict__ f, unsigned V, unsigned x, float2 v[3])
{
    if (PAIRS) {
        const float4 p = reinterpret_cast<const float4 *>(f)[x];
        v[0] = make_float2(p.x, p.y);
        v[1] = make_float2(p.z, p.w);
        v[2] = f[2 * V + x];
    } else {
#pragma unroll
        for (int q = 0; q < 3; q++) v[q] = f[q * V + x];
    }
}

template <bool PAIRS>
__device__ __forceinline__ void store_site(float2 *__restrict__ o, unsigned V, unsigned x, const float2 v[3])
{
    if (PAIRS) {
        reinterpret_cast<float4 *>(o)[x] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
        o[2 * V + x] = v[2];
    } else {
#pragma unroll
        for (int q = 0; q < 3; q++) o[q * V + x] = v[q];
    }
}

// The first NE entries of the link of direction block um at site x.
template <bool PAIRS, int NE>
__device__ __forceinline__ void load_link(const float2 *__restrict__ um, unsigned V, unsigned x, float2 u[9])
{
    if (PAIRS) {
#pragma unroll
        for (int b = 0; 2 * b + 1 < NE; b++) {
#if LAP_SOA_LINKS_CG
            const float4 p = __ldcg(reinterpret_cast<const float4 *>(um + 2 * b * V) + x);
#else
            const float4 p = __ldg(reinterpret_cast<const float4 *>(um + 2 * b * V) + x);
#endif
            u[2 * b] = make_float2(p.x, p.y);
            u[2 * b + 1] = make_float2(p.z, p.w);
        }
        if (NE == 9) u[8] = __ldg(um + 8 * V + x);
    } else {
#pragma unroll
        for (int k = 0; k < NE; k++) {
#if LAP_SOA_LINKS_CG
            u[k] = __ldcg(um + k * V + x);
#else
            u[k] = __ldg(um + k * V + x);
#endif
        }
    }
}

// The transpose of the links runs once per solve; it sets *bad when a link's
// third row differs from the one rebuilt from its first two by more than tol
// (the links are not SU(3) to FP32 accuracy), in which case the stencil reads
// all three rows.
constexpr float SU3_TOL = 2e-6f;
template <bool PAIRS>
__global__ void links_soa_kernel(const float2 *__restrict__ U, float2 *__restrict__ Us, unsigned V,
                                 int *__restrict__ bad)
{
    const int t = blockIdx.y;
    const unsigned x = blockIdx.x * blockDim.x + threadIdx.x;
    bool off = false;
    if (x < V) {
        const float2 *u = U + (long long)t * 27 * V;
        float2 *o = Us + (long long)t * 27 * V;
#pragma unroll
        for (int mu = 0; mu < 3; mu++) {
            float2 m[9];
#pragma unroll
            for (int rc = 0; rc < 9; rc++) m[rc] = u[((long long)mu * V + x) * 9 + rc];
            float2 *om = o + (long long)mu * 9 * V;
            if (PAIRS) {
#pragma unroll
                for (int b = 0; b < 4; b++)
                    reinterpret_cast<float4 *>(om + 2 * b * V)[x] =
                        make_float4(m[2 * b].x, m[2 * b].y, m[2 * b + 1].x, m[2 * b + 1].y);
                om[8 * V + x] = m[8];
            } else {
#pragma unroll
                for (int rc = 0; rc < 9; rc++) om[(long long)rc * V + x] = m[rc];
            }
            float2 r[9];
#pragma unroll
            for (int k = 0; k < 6; k++) r[k] = m[k];
            su3_third_row(r);
#pragma unroll
            for (int k = 6; k < 9; k++) off |= !(fabsf(r[k].x - m[k].x) <= SU3_TOL && fabsf(r[k].y - m[k].y) <= SU3_TOL);
        }
    }
    if (__ballot_sync(0xffffffffu, off) && (threadIdx.x & 31) == 0) atomicOr(bad, 1);
}

// lap_kernel in the solver's layouts: out = a (-Delta in) + b in + c z.
// Launched as a programmatic dependent of the previous step (a filter step
// reads its predecessors' outputs and overwrites the vector read two steps
// back): it lets the next grid be scheduled at once and waits for the full
// completion of the previous grid before its first access to vectors.
// R12: the links are SU(3) and only their first two rows are read.  PAIRS:
// the paired layouts above.
template <bool R12, bool PAIRS>
__global__ void __launch_bounds__(LAP_SOA_THREADS, LAP_SOA_MINB) lap_soa_kernel(const float2 *__restrict__ Us,
                                                              const float2 *__restrict__ in,
                                                              const float2 *__restrict__ z, float2 *__restrict__ out,
                                                              int L, long long ts_in, long long ts_z, long long ts_out,
                                                              float a, float b, float c)
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    // offsets within a timeslice are 32-bit (L <= 512: 9 V < 2^31); two
    // 32-bit divisions give the coordinates
    const unsigned uL = (unsigned)L, V = uL * uL * uL;
    const unsigned x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= V) return;
    const int n = blockIdx.y, t = blockIdx.z;
    const float2 *f = in + t * ts_in + (long long)n * V * 3;
    const float2 *Ut = Us + (long long)t * 27 * V;
    const unsigned q1 = x / uL, c0 = x - q1 * uL, c2 = q1 / uL, c1 = q1 - c2 * uL;
    const unsigned cc[3] = {c0, c1, c2};
    const unsigned stride[3] = {1u, uL, uL * uL};
    float2 fx[3], acc[3];
    load_site<PAIRS>(f, V, x, fx);
#pragma unroll
    for (int q = 0; q < 3; q++) acc[q] = make_float2(0.f, 0.f);
#pragma unroll
    for (int mu = 0; mu < 3; mu++) {
        const unsigned up = cc[mu] == uL - 1 ? x - (uL - 1) * stride[mu] : x + stride[mu];
        const unsigned dn = cc[mu] == 0 ? x + (uL - 1) * stride[mu] : x - stride[mu];
        const float2 *um = Ut + (long long)mu * 9 * V;
        // all loads of this direction issued before its multiply-adds
        float2 fu[3], fd[3], uf[9], ub[9];
        load_site<PAIRS>(f, V, up, fu);
        load_site<PAIRS>(f, V, dn, fd);
        load_link<PAIRS, R12 ? 6 : 9>(um, V, x, uf);
        load_link<PAIRS, R12 ? 6 : 9>(um, V, dn, ub);
        if (R12) {
            su3_third_row(uf);
            su3_third_row(ub);
        }
#pragma unroll
        for (int r = 0; r < 3; r++)
#pragma unroll
            for (int q = 0; q < 3; q++) {
                acc[r] = cfma(uf[3 * r + q], fu[q], acc[r]);          // U_mu(x)_{rq} f_q(x + mu)
                acc[r] = cfma_conj(ub[3 * q + r], fd[q], acc[r]);     // conj(U_mu(x - mu)_{qr}) f_q(x - mu)
            }
    }
    float2 *o = out + t * ts_out + (long long)n * V * 3;
    float2 zv[3] = {};
    if (z) load_site<PAIRS>(z + t * ts_z + (long long)n * V * 3, V, x, zv);
    float2 r[3];
#pragma unroll
    for (int q = 0; q < 3; q++) {
        const float2 lap = make_float2(6.f * fx[q].x - acc[q].x, 6.f * fx[q].y - acc[q].y);
        r[q] = make_float2(a * lap.x + b * fx[q].x + c * zv[q].x, a * lap.y + b * fx[q].y + c * zv[q].y);
    }
    store_site<PAIRS>(o, V, x, r);
}

// Block reduction of a double into thread 0.
__device__ __forceinline__ double block_sum(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    v = 0.0;
    if (threadIdx.x < (blockDim.x >> 5)) v = sh[threadIdx.x];
    if (w == 0)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Gram-Schmidt inner products, dots[t][j] += <basis[t][j], w[t]> over this
// block's elements, j < nj.  Each thread holds DOT_EPT elements of w in
// registers; per row the products are summed in FP32 within the thread and
// the warp (shuffles), the warps' partials in FP64 and across blocks with
// FP64 atomics.  GB300's FP64 rate is a small fraction of its FP32 rate, so no
// FP64 arithmetic runs per element.
constexpr int DOT_EPT = 8;      // elements of w per thread
constexpr int DOT_JC = 32;      // rows between flushes of the warp partials
constexpr int DOT_RG = 4;       // rows whose loads are issued together
__global__ void __launch_bounds__(LAP_THREADS) dots_kernel(const float2 *__restrict__ basis, long long ts_basis,
                                                           const float2 *__restrict__ w, long long ts_w, long long K,
                                                           int nj, double2 *__restrict__ dots, int dots_stride)
{
    __shared__ float2 part[LAP_THREADS / 32][DOT_JC];
    const int t = blockIdx.y, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long e0 = (long long)blockIdx.x * LAP_THREADS * DOT_EPT + threadIdx.x;
    const float2 *B = basis + t * ts_basis;
    float2 wv[DOT_EPT];
#pragma unroll
    for (int q = 0; q < DOT_EPT; q++) {
        const long long e = e0 + (long long)q * LAP_THREADS;
        wv[q] = e < K ? w[t * ts_w + e] : make_float2(0.f, 0.f);
    }
    for (int j0 = 0; j0 < nj; j0 += DOT_JC) {
        const int jn = min(DOT_JC, nj - j0);
        for (int jj = 0; jj < jn; jj += DOT_RG) {
            float2 b[DOT_RG][DOT_EPT];
#pragma unroll
            for (int r = 0; r < DOT_RG; r++)
#pragma unroll
                for (int q = 0; q < DOT_EPT; q++) {
                    const long long e = e0 + (long long)q * LAP_THREADS;
                    b[r][q] = (jj + r < jn && e < K) ? B[(long long)(j0 + jj + r) * K + e] : make_float2(0.f, 0.f);
                }
#pragma unroll
            for (int r = 0; r < DOT_RG; r++) {
                float re = 0.f, im = 0.f;
#pragma unroll
                for (int q = 0; q < DOT_EPT; q++) {
                    re = fmaf(b[r][q].x, wv[q].x, fmaf(b[r][q].y, wv[q].y, re));
                    im = fmaf(b[r][q].x, wv[q].y, fmaf(-b[r][q].y, wv[q].x, im));
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    re += __shfl_xor_sync(0xffffffffu, re, o);
                    im += __shfl_xor_sync(0xffffffffu, im, o);
                }
                if (lane == 0 && jj + r < jn) part[warp][jj + r] = make_float2(re, im);
            }
        }
        __syncthreads();
        if (threadIdx.x < jn) {
            double re = 0.0, im = 0.0;
#pragma unroll
            for (int q = 0; q < LAP_THREADS / 32; q++) {
                re += part[q][threadIdx.x].x;
                im += part[q][threadIdx.x].y;
            }
            atomicAdd(&dots[t * dots_stride + j0 + threadIdx.x].x, re);
            atomicAdd(&dots[t * dots_stride + j0 + threadIdx.x].y, im);
        }
        __syncthreads();
    }
}

// Gram-Schmidt update, w[t] -= sum_j coef[t][j] basis[t][j] for j < nj, with
// the coefficients rounded to FP32 in shared memory (dynamic, nj float2) and
// FP32 multiply-adds; UPD_EPT elements per thread, the loads of UPD_RG rows
// issued together.  norm (may be null): norm[t] += |w[t]|^2 of the result.
constexpr int UPD_EPT = 4;
constexpr int UPD_RG = 4;
__global__ void __launch_bounds__(LAP_THREADS) update_kernel(const float2 *__restrict__ basis, long long ts_basis,
                                                             float2 *__restrict__ w, long long ts_w, long long K, int nj,
                                                             const double2 *__restrict__ coef, int coef_stride,
                                                             double *__restrict__ norm)
{
    extern __shared__ float2 cs[];
    __shared__ float npart[LAP_THREADS / 32];
    const int t = blockIdx.y;
    for (int i = threadIdx.x; i < nj; i += LAP_THREADS) {
        const double2 c = coef[t * coef_stride + i];
        cs[i] = make_float2((float)c.x, (float)c.y);
    }
    __syncthreads();
    const long long e0 = (long long)blockIdx.x * LAP_THREADS * UPD_EPT + threadIdx.x;
    const float2 *B = basis + t * ts_basis;
    float2 acc[UPD_EPT];
#pragma unroll
    for (int q = 0; q < UPD_EPT; q++) acc[q] = make_float2(0.f, 0.f);
    for (int j = 0; j < nj; j += UPD_RG) {
        float2 b[UPD_RG][UPD_EPT];
#pragma unroll
        for (int r = 0; r < UPD_RG; r++)
#pragma unroll
            for (int q = 0; q < UPD_EPT; q++) {
                const long long e = e0 + (long long)q * LAP_THREADS;
                b[r][q] = (j + r < nj && e < K) ? B[(long long)(j + r) * K + e] : make_float2(0.f, 0.f);
            }
#pragma unroll
        for (int r = 0; r < UPD_RG; r++) {
            const float2 c = j + r < nj ? cs[j + r] : make_float2(0.f, 0.f);
#pragma unroll
            for (int q = 0; q < UPD_EPT; q++) acc[q] = cfma(c, b[r][q], acc[q]);
        }
    }
    float nrm = 0.f;
#pragma unroll
    for (int q = 0; q < UPD_EPT; q++) {
        const long long e = e0 + (long long)q * LAP_THREADS;
        if (e < K) {
            float2 &x = w[t * ts_w + e];
            const float2 v = make_float2(x.x - acc[q].x, x.y - acc[q].y);
            x = v;
            nrm = fmaf(v.x, v.x, fmaf(v.y, v.y, nrm));
        }
    }
    if (norm) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
        if ((threadIdx.x & 31) == 0) npart[threadIdx.x >> 5] = nrm;
        __syncthreads();
        if (threadIdx.x == 0) {
            double sum = 0.0;
            for (int q = 0; q < LAP_THREADS / 32; q++) sum += npart[q];
            atomicAdd(&norm[t], sum);
        }
    }
}

// out[t] = w[t] * scale[t] (scale per timeslice, FP64).
// copy: a second destination (may be null), [T][K].
__global__ void scale_kernel(const float2 *__restrict__ w, long long ts_w, float2 *__restrict__ out, long long ts_out,
                             long long K, const double *__restrict__ scale, float2 *__restrict__ copy)
{
    const int t = blockIdx.y;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= K) return;
    const float s = (float)scale[t];
    const float2 v = w[t * ts_w + e];
    const float2 r = make_float2(v.x * s, v.y * s);
    out[t * ts_out + e] = r;
    if (copy) copy[t * K + e] = r;
}

// alpha[t][j] = Re <v_j, A v_j>: row j of the first Gram-Schmidt pass's
// coefficients (dots, [T][ld]).
__global__ void take_alpha_kernel(const double2 *__restrict__ dots, int ld, int j, double *__restrict__ alpha, int m,
                                  int T)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < T) alpha[(long long)t * m + j] = dots[(long long)t * ld + j].x;
}

// beta[t][j] = |w| after both Gram-Schmidt passes (norm2 = |w|^2), the scale
// 1/|w| of the next basis vector, and in *brk the earliest step at which |w|
// fell below 1e-6 max(1, |alpha|) (an invariant subspace; only when check).
__global__ void take_beta_kernel(const double *__restrict__ norm2, const double *__restrict__ alpha, int j, int m,
                                 int T, int check, double *__restrict__ beta, double *__restrict__ scale,
                                 int *__restrict__ brk)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    const double a = alpha[(long long)t * m + j], b = sqrt(fmax(norm2[t], 0.0));
    beta[(long long)t * m + j] = b;
    scale[t] = b > 1e-30 ? 1.0 / b : 0.0;
    if (check && b < 1e-6 * fmax(1.0, fabs(a))) atomicMin(brk, j);
}

// X[t][r] = sum_j S[t][j][r] basis[t][j] for r < nr (S real, [T][m][nr]); each
// thread one element and RT outputs, the S column block staged in shared memory.
constexpr int RT = 16;
__global__ void __launch_bounds__(LAP_THREADS) ritz_kernel(const float2 *__restrict__ basis, long long ts_basis,
                                                           long long K, int m, const double *__restrict__ S, int nr,
                                                           float2 *__restrict__ X, long long ts_X)
{
    __shared__ float Ss[64][RT];
    const int t = blockIdx.y, r0 = blockIdx.z * RT;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float2 acc[RT];
#pragma unroll
    for (int r = 0; r < RT; r++) acc[r] = make_float2(0.f, 0.f);
    for (int j0 = 0; j0 < m; j0 += 64) {
        __syncthreads();
        for (int i = threadIdx.x; i < 64 * RT; i += blockDim.x) {
            const int jj = j0 + i / RT, rr = r0 + i % RT;
            Ss[i / RT][i % RT] = (jj < m && rr < nr) ? (float)S[((long long)t * m + jj) * nr + rr] : 0.f;
        }
        __syncthreads();
        if (e < K) {
            const int jn = min(64, m - j0);
            for (int jj = 0; jj < jn; jj++) {
                const float2 b = basis[t * ts_basis + (long long)(j0 + jj) * K + e];
#pragma unroll
                for (int r = 0; r < RT; r++) {
                    acc[r].x = fmaf(Ss[jj][r], b.x, acc[r].x);
                    acc[r].y = fmaf(Ss[jj][r], b.y, acc[r].y);
                }
            }
        }
    }
    if (e >= K) return;
#pragma unroll
    for (int r = 0; r < RT; r++)
        if (r0 + r < nr) X[t * ts_X + (long long)(r0 + r) * K + e] = acc[r];
}

// Per (timeslice, vector) sums over the elements: xy = <x, y>, xx = <x, x>
// (mode 0), or rr = |y - lam x|^2 (mode 1, lam per vector).
__global__ void __launch_bounds__(LAP_THREADS) rayleigh_kernel(const float2 *__restrict__ X, const float2 *__restrict__ Y,
                                                               long long ts, long long K, int mode,
                                                               const double *__restrict__ lam, int nr,
                                                               double *__restrict__ out)
{
    __shared__ double sh[LAP_THREADS / 32];
    const int t = blockIdx.y, r = blockIdx.z;
    const float2 *x = X + t * ts + (long long)r * K, *y = Y + t * ts + (long long)r * K;
    double s0 = 0.0, s1 = 0.0;
    const double l = mode ? lam[t * nr + r] : 0.0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < K; e += (long long)gridDim.x * blockDim.x) {
        const float2 a = x[e], b = y[e];
        if (mode == 0) {
            s0 += (double)a.x * b.x + (double)a.y * b.y;
            s1 += (double)a.x * a.x + (double)a.y * a.y;
        } else {
            const double dx = b.x - l * a.x, dy = b.y - l * a.y;
            s0 += dx * dx + dy * dy;
        }
    }
    s0 = block_sum(s0, sh);
    s1 = block_sum(s1, sh);
    if (threadIdx.x == 0) {
        atomicAdd(&out[2 * (t * nr + r)], s0);
        atomicAdd(&out[2 * (t * nr + r) + 1], s1);
    }
}

// out[t][r] = X[t][perm[t][r]] * scale[t][r], from the solver's vector
// layout to the caller's [V][3].
template <bool PAIRS>
__global__ void gather_kernel(const float2 *__restrict__ X, long long ts_X, const int *__restrict__ perm,
                              const double *__restrict__ scale, int nr, float2 *__restrict__ out, long long ts_out,
                              long long V)
{
    const int t = blockIdx.y, r = blockIdx.z;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 3 * V) return;
    const long long x = e / 3;
    const int q = (int)(e - 3 * x);
    const float sc = (float)scale[t * nr + r];
    const long long src = PAIRS ? (q < 2 ? 2 * x + q : 2 * V + x) : q * V + x;
    const float2 v = X[t * ts_X + (long long)perm[t * nr + r] * 3 * V + src];
    out[t * ts_out + (long long)r * 3 * V + e] = make_float2(v.x * sc, v.y * sc);
}

}  // namespace

// Length of the vector (a, b): the plain formula while the squares can neither
// overflow nor underflow, std::hypot outside that range.
static inline double norm2(double a, double b)
{
    const double m = std::max(std::fabs(a), std::fabs(b));
    return (m > 1e-150 && m < 1e150) ? std::sqrt(a * a + b * b) : std::hypot(a, b);
}

// One implicit symmetric QR step with a Wilkinson shift on the unreduced block
// [lo, hi] of the tridiagonal matrix (diagonal a, off-diagonal b; b[i] couples
// i and i+1), after Golub and Van Loan, "Matrix Computations", the implicit
// symmetric QR step: the shift mu is the eigenvalue of the trailing 2 x 2 of
// the block nearer to its last diagonal entry; the first rotation is the one
// that zeroes the second entry of the first column of (T - mu I), and the
// bulge it creates below the subdiagonal is chased down the block by one
// rotation per row.  Rotation k acts on rows and columns k, k+1 as
// Q = [[c, -s], [s, c]]; every rotation is applied to the rows k, k+1 of zt,
// the transpose of the eigenvector matrix.
static void qr_step(int lo, int hi, double *a, double *b, double *zt, int n)
{
    const double delta = 0.5 * (a[hi - 1] - a[hi]);
    const double bt = b[hi - 1];
    const double den = delta + (delta >= 0.0 ? 1.0 : -1.0) * norm2(delta, bt);
    const double mu = a[hi] - bt * (bt / den);
    double x = a[lo] - mu;   // entry kept by the next rotation
    double y = b[lo];        // entry it annihilates
    for (int k = lo; k < hi; k++) {
        const double r = norm2(x, y);
        double c = 1.0, s = 0.0;
        if (r > 0.0) {
            c = x / r;
            s = y / r;
        }
        if (k > lo) b[k - 1] = r;   // the bulge below it is gone
        const double ak = a[k], ak1 = a[k + 1], bk = b[k];
        const double cc = c * c, ss = s * s, cs = c * s;
        a[k] = cc * ak + 2.0 * cs * bk + ss * ak1;
        a[k + 1] = ss * ak + ak1 * cc - 2.0 * cs * bk;
        b[k] = cs * (ak1 - ak) + (cc - ss) * bk;
        if (k + 1 < hi) {
            // the rotation of columns k, k+1 carries b[k+1] into row k+2, column k
            x = b[k];
            y = s * b[k + 1];
            b[k + 1] *= c;
        }
        double *u = zt + (size_t)k * n, *v = u + n;
        for (int j = 0; j < n; j++) {
            const double uj = u[j], vj = v[j];
            u[j] = c * uj + s * vj;
            v[j] = c * vj - s * uj;
        }
    }
}

// Eigenvalues d (ascending) and orthonormal eigenvectors z (column k of the n x n
// row-major z belongs to d[k]) of the symmetric tridiagonal matrix with diagonal
// d[0..n) and off-diagonal e[0..n-1), by the symmetric QR algorithm: off-diagonal
// entries below DBL_EPSILON times their two diagonal neighbours are set to zero,
// and the lowest unreduced block that is left takes one implicit QR step, until
// the matrix is diagonal.  Returns 0, or -1 after 60 n steps without
// convergence.
int tridiag_eigen(int n, double *d, const double *e_in, double *z)
{
    std::vector<double> b(n > 1 ? n - 1 : 1, 0.0), zt((size_t)n * n, 0.0);
    for (int i = 0; i + 1 < n; i++) b[i] = e_in[i];
    for (int i = 0; i < n; i++) zt[(size_t)i * n + i] = 1.0;
    const double eps = std::numeric_limits<double>::epsilon();
    long long steps = 0;
    int hi = n - 1;
    while (hi > 0) {
        for (int i = 0; i < hi; i++)
            if (std::fabs(b[i]) <= eps * (std::fabs(d[i]) + std::fabs(d[i + 1])) ||
                std::fabs(b[i]) < std::numeric_limits<double>::min())
                b[i] = 0.0;
        while (hi > 0 && b[hi - 1] == 0.0) hi--;   // trailing entries already diagonal
        if (hi == 0) break;
        int lo = hi - 1;
        while (lo > 0 && b[lo - 1] != 0.0) lo--;
        if (++steps > 60LL * n) return -1;
        qr_step(lo, hi, d, b.data(), zt.data(), n);
    }
    // ascending order
    std::vector<int> idx(n);
    for (int i = 0; i < n; i++) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int x, int y) { return d[x] < d[y]; });
    std::vector<double> d2(n);
    for (int k = 0; k < n; k++) {
        d2[k] = d[idx[k]];
        const double *col = zt.data() + (size_t)idx[k] * n;
        for (int i = 0; i < n; i++) z[(size_t)i * n + k] = col[i];
    }
    std::memcpy(d, d2.data(), sizeof(double) * n);
    return 0;
}

cudaError_t launch_laplacian(const float2 *U, const float2 *in, const float2 *z, float2 *out, int L, int T, int nvec,
                             long long ts_in, long long ts_z, long long ts_out, float a, float b, float c, cudaStream_t s)
{
    const long long V = (long long)L * L * L;
    if (T > 65535 || nvec > 65535) return cudaErrorInvalidValue;
    dim3 g((unsigned)((V + LAP_THREADS - 1) / LAP_THREADS), (unsigned)nvec, (unsigned)T);
    lap_kernel<<<g, LAP_THREADS, 0, s>>>(U, in, z, out, L, ts_in, ts_z, ts_out, a, b, c);
    return cudaGetLastError();
}

cudaError_t launch_lap_soa(const float2 *Us, const float2 *in, const float2 *z, float2 *out, int L, int T, int nvec,
                           long long ts_in, long long ts_z, long long ts_out, float a, float b, float c, cudaStream_t s,
                           bool r12, bool pairs, bool pdl = false)
{
    const long long V = (long long)L * L * L;
    if (T > 65535 || nvec > 65535) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((V + LAP_SOA_THREADS - 1) / LAP_SOA_THREADS), (unsigned)nvec, (unsigned)T);
    cfg.blockDim = dim3(LAP_SOA_THREADS);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    if (pairs)
        return r12 ? cudaLaunchKernelEx(&cfg, lap_soa_kernel<true, true>, Us, in, z, out, L, ts_in, ts_z, ts_out, a, b, c)
                   : cudaLaunchKernelEx(&cfg, lap_soa_kernel<false, true>, Us, in, z, out, L, ts_in, ts_z, ts_out, a, b, c);
    return r12 ? cudaLaunchKernelEx(&cfg, lap_soa_kernel<true, false>, Us, in, z, out, L, ts_in, ts_z, ts_out, a, b, c)
               : cudaLaunchKernelEx(&cfg, lap_soa_kernel<false, false>, Us, in, z, out, L, ts_in, ts_z, ts_out, a, b, c);
}

}  // namespace laph

using namespace laph;

#define LCK(call)                                                   \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) {                                    \
            rc = laph::record_cuda_error(e_, #call);                \
            goto done;                                              \
        }                                                           \
    } while (0)

extern "C" {

int laph_laplacian(const void *U, const void *f, void *out, int L, int T, int nvec, void *stream)
{
    if (!U || !f || !out || L < 2 || L > 1024 || T < 1 || T > 65535 || nvec < 1 || nvec > 65535) return LAPH_ERR_ARG;
    if (((uintptr_t)U | (uintptr_t)f | (uintptr_t)out) % 8) return LAPH_ERR_ARG;
    const long long V = (long long)L * L * L;
    cudaError_t e = launch_laplacian((const float2 *)U, (const float2 *)f, nullptr, (float2 *)out, L, T, nvec,
                                     (long long)nvec * V * 3, 0, (long long)nvec * V * 3, 1.f, 0.f, 0.f,
                                     (cudaStream_t)stream);
    return e == cudaSuccess ? LAPH_OK : laph::record_cuda_error(e, "laplacian");
}

int laph_tridiag_eigen(int n, double *d, const double *e, double *z)
{
    if (n < 1 || !d || (!e && n > 1) || !z) return LAPH_ERR_ARG;
    return laph::tridiag_eigen(n, d, e, z) == 0 ? LAPH_OK : LAPH_ERR_ARG;
}

}  // extern "C"

namespace {

// Device workspace of one solve, offsets 256-byte aligned.  The basis holds
// m + 1 vectors of every timeslice; after the Ritz vectors have been formed it
// is reused for (-Delta) applied to them.
struct LzLayout {
    size_t Us, basis, w, ya, yb, yc, vin, X, dots, dscale, dnorm, dS, dred, dlam, dperm, dflag, dalpha, dbeta, dbrk,
        total;
};

LzLayout lz_layout(long long K, int T, int m, int nr)
{
    LzLayout l{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    };
    l.Us = take(sizeof(float2) * (size_t)9 * K * T);
    l.basis = take(sizeof(float2) * (size_t)K * (m + 1) * T);
    l.w = take(sizeof(float2) * (size_t)K * T);
    l.ya = take(sizeof(float2) * (size_t)K * T);
    l.yb = take(sizeof(float2) * (size_t)K * T);
    l.yc = take(sizeof(float2) * (size_t)K * T);
    l.vin = take(sizeof(float2) * (size_t)K * T);
    l.X = take(sizeof(float2) * (size_t)K * nr * T);
    l.dots = take(sizeof(double2) * (size_t)(m + 1) * T);
    l.dscale = take(sizeof(double) * T);
    l.dnorm = take(sizeof(double) * T);
    l.dS = take(sizeof(double) * (size_t)T * m * nr);
    l.dred = take(sizeof(double) * 2 * (size_t)T * nr);
    l.dlam = take(sizeof(double) * (size_t)T * nr);
    l.dperm = take(sizeof(int) * (size_t)T * nr);
    l.dflag = take(sizeof(int));
    l.dalpha = take(sizeof(double) * (size_t)T * m);
    l.dbeta = take(sizeof(double) * (size_t)T * m);
    l.dbrk = take(sizeof(int));
    l.total = off;
    return l;
}

int lz_check(int L, int T, int n_ev, const laph_lanczos_params *prm)
{
    if (!prm || L < 2 || L > 512 || T < 1 || T > 65535 || n_ev < 1) return LAPH_ERR_ARG;
    const long long K = 3LL * L * L * L;
    const int m = prm->n_krylov;
    if (m < n_ev || m > 4096 || (long long)m > K || prm->cheb_degree < 0 || prm->cheb_degree > 10000) return LAPH_ERR_ARG;
    if (prm->cheb_degree > 0 && !(prm->cheb_lo > 0.0 && prm->cheb_lo < 12.0)) return LAPH_ERR_ARG;
    if (prm->ts_group < 0) return LAPH_ERR_ARG;
    if (prm->link_rows != 0 && prm->link_rows != 2 && prm->link_rows != 3) return LAPH_ERR_ARG;
    return LAPH_OK;
}

}  // namespace

extern "C" {

int laph_lanczos_workspace_size(int L, int T, int n_ev, const laph_lanczos_params *prm, size_t *bytes)
{
    if (!bytes) return LAPH_ERR_ARG;
    const int rc = lz_check(L, T, n_ev, prm);
    if (rc != LAPH_OK) return rc;
    *bytes = lz_layout(3LL * L * L * L, T, prm->n_krylov, n_ev).total;
    return LAPH_OK;
}

int laph_lanczos(const void *U, int L, int T, int n_ev, const laph_lanczos_params *prm, void *evecs, double *evals,
                 double *resid, void *workspace, size_t workspace_bytes, laph_lanczos_stats *stats, void *stream)
{
    if (!U || !evecs || !evals) return LAPH_ERR_ARG;
    int rc = lz_check(L, T, n_ev, prm);
    if (rc != LAPH_OK) return rc;
    if (((uintptr_t)U | (uintptr_t)evecs) % 8) return LAPH_ERR_ARG;
    const long long V = (long long)L * L * L, K = 3 * V;
    const int m = prm->n_krylov, nr = n_ev, d = prm->cheb_degree;
    const LzLayout lay = lz_layout(K, T, m, nr);
    if (workspace && (workspace_bytes < lay.total || (uintptr_t)workspace % 256)) return LAPH_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    char *ws = (char *)workspace, *owned = nullptr;
    cudaEvent_t ev[7] = {};   // call start, loop start, iteration (apply, orth, end), loop end, call end
    std::vector<cudaEvent_t> step_ev;   // with stats: per Krylov step without host synchronisation, apply start,
                                        // apply end, orthogonalisation end
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t filter = nullptr;
    laph_lanczos_stats st = {};
    const long long ts_b = (long long)(m + 1) * K;   // basis of one timeslice
    std::vector<double> alpha((size_t)T * m, 0.0), beta((size_t)T * m, 0.0), h_dots(2 * (size_t)T * (m + 1)),
        h_norm(T), h_scale(T), h_S((size_t)T * m * nr, 0.0), h_red(2 * (size_t)T * nr);
    const unsigned blocks_e = (unsigned)((K + LAP_THREADS - 1) / LAP_THREADS);
    const unsigned blocks_dot = (unsigned)((K + LAP_THREADS * DOT_EPT - 1) / (LAP_THREADS * DOT_EPT));
    const unsigned blocks_upd = (unsigned)((K + LAP_THREADS * UPD_EPT - 1) / (LAP_THREADS * UPD_EPT));
    const double cheb_c = 0.5 * (12.0 + prm->cheb_lo), cheb_e = 0.5 * (12.0 - prm->cheb_lo);
    // filter steps run group by group of timeslices, so that a group's links
    // and the five vectors the recurrence touches, 8 (27 + 15) V bytes per
    // timeslice, stay in L2 across its d steps: groups filling about 70% of the
    // L2 (measured at L = 32, T = 64 on GB300: 8 timeslices, 88 MB, take 0.71x
    // the time of one group of all 64; 16 timeslices overflow it)
    int tg = prm->ts_group, dev = 0, l2 = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess)
        l2 = 0;
    if (tg == 0) tg = (int)std::max<long long>(1, (long long)(0.7 * l2) / (8 * 42 * V));
    tg = std::min(tg, T);
    // SU(3) links can be read as two rows (the third rebuilt), 144 instead of
    // 216 bytes per site: a gain where the stencil streams them from HBM
    // (measured at L = 32, T = 64 on GB300: 0.83x the filter time), a loss
    // where a filter group's links stay in L2 (1.04x).  Automatic choice: two
    // rows unless the filter runs in groups that fit in L2.
    const bool group_in_l2 = d > 0 && (double)tg * 8 * 42 * V <= 0.7 * l2;
    st.ts_group = d > 0 ? tg : T;
    const bool want_r12 = prm->link_rows == 2 || (prm->link_rows == 0 && !group_in_l2);
    const bool pdl = prm->pdl != 0;
    bool r12 = false;
    // paired layouts where every block they split into is 16-byte aligned
    const bool pairs = V % 2 == 0;
    float2 *Ud, *basis, *w, *ya, *yb, *yc, *vin, *X, *Y;
    double2 *dots;
    double *dscale, *dnorm, *dS, *dred, *dlam, *dalpha, *dbeta;
    int *dperm, *dbrk;

    if (stats) {
        for (auto &e : ev) LCK(cudaEventCreate(&e));
        step_ev.assign(3 * (size_t)m, nullptr);
        for (auto &e : step_ev) LCK(cudaEventCreate(&e));
        LCK(cudaEventRecord(ev[0], s));
    }
    if (!ws) {
        LCK(cudaMallocAsync((void **)&owned, lay.total, s));
        ws = owned;
    }
    Ud = (float2 *)(ws + lay.Us);
    basis = (float2 *)(ws + lay.basis);
    w = (float2 *)(ws + lay.w);
    ya = (float2 *)(ws + lay.ya);
    yb = (float2 *)(ws + lay.yb);
    yc = (float2 *)(ws + lay.yc);
    vin = (float2 *)(ws + lay.vin);
    X = (float2 *)(ws + lay.X);
    Y = basis;
    dots = (double2 *)(ws + lay.dots);
    dscale = (double *)(ws + lay.dscale);
    dnorm = (double *)(ws + lay.dnorm);
    dS = (double *)(ws + lay.dS);
    dred = (double *)(ws + lay.dred);
    dlam = (double *)(ws + lay.dlam);
    dperm = (int *)(ws + lay.dperm);
    dalpha = (double *)(ws + lay.dalpha);
    dbeta = (double *)(ws + lay.dbeta);
    dbrk = (int *)(ws + lay.dbrk);

    {
        // the operator on the newest basis vector v (of every timeslice) -> w
        // The Chebyshev filter of the vectors in vin (stride K) into w on stream
        // cs.  Recurrence in B = (A - c) / e:
        //   y_0 = v, y_1 = B v, y_{k+1} = 2 B y_k - y_{k-1}, result y_d in w;
        // three scratch vectors rotate, so no step writes an operand it reads.
        // All d steps of a group of timeslices run before the next group's.
        auto filter_launches = [&](cudaStream_t cs) -> cudaError_t {
            cudaError_t e = cudaSuccess;
            const float2 *v = vin;
            const long long ts_v = K;
            for (int t0 = 0; t0 < T && e == cudaSuccess; t0 += tg) {
                const int nt = std::min(tg, T - t0);
                const float2 *Ug = Ud + (long long)t0 * 27 * V;
                auto at = [&](const float2 *base, long long ts) { return base + (long long)t0 * ts; };
                float2 *y1 = d == 1 ? w : ya;
                e = launch_lap_soa(Ug, at(v, ts_v), nullptr, (float2 *)at(y1, K), L, nt, 1, ts_v, 0, K,
                                     (float)(1.0 / cheb_e), (float)(-cheb_c / cheb_e), 0.f, cs, r12, pairs, pdl && t0 > 0);
                const float2 *prev = v;
                long long ts_prev = ts_v;
                float2 *cur = y1;
                for (int k = 2; k <= d && e == cudaSuccess; k++) {
                    float2 *dst = k == d ? w : (cur != ya && prev != ya ? ya : (cur != yb && prev != yb ? yb : yc));
                    e = launch_lap_soa(Ug, at(cur, K), at(prev, ts_prev), (float2 *)at(dst, K), L, nt, 1, K, ts_prev,
                                         K, (float)(2.0 / cheb_e), (float)(-2.0 * cheb_c / cheb_e), -1.f, cs, r12, pairs, pdl);
                    prev = cur;
                    ts_prev = K;
                    cur = dst;
                }
            }
            return e;
        };
        const int n_filter = d * ((T + tg - 1) / tg);
        // the operator on the newest basis vector v (of every timeslice) -> w; for
        // the filter v is also in vin, and its launches replay as one CUDA graph
        auto apply = [&](const float2 *v) -> cudaError_t {
            if (d == 0) {
                st.launches++;
                st.apply_launches++;
                return launch_lap_soa(Ud, v, nullptr, w, L, T, 1, ts_b, 0, K, 1.f, 0.f, 0.f, s, r12, pairs);
            }
            st.launches += n_filter;
            st.apply_launches += n_filter;
            if (filter) return cudaGraphLaunch(filter, s);
            return filter_launches(s);
        };
        // removes from w its components along basis vectors [0, nj), twice
        // ("twice is enough"); the first pass's coefficients land in h_dots,
        // |w|^2 of the result in h_norm.  Synchronises the stream.
        auto orthogonalise = [&](int nj) -> cudaError_t {
            cudaError_t e = cudaSuccess;
            for (int pass = 0; pass < 2 && e == cudaSuccess; pass++) {
                e = cudaMemsetAsync(dots, 0, sizeof(double2) * (m + 1) * T, s);
                if (e == cudaSuccess && pass == 1) e = cudaMemsetAsync(dnorm, 0, sizeof(double) * T, s);
                if (e != cudaSuccess) break;
                dots_kernel<<<dim3(blocks_dot, T), LAP_THREADS, 0, s>>>(basis, ts_b, w, K, K, nj, dots, m + 1);
                update_kernel<<<dim3(blocks_upd, T), LAP_THREADS, sizeof(float2) * nj, s>>>(
                    basis, ts_b, w, K, K, nj, dots, m + 1, pass == 1 ? dnorm : nullptr);
                e = cudaGetLastError();
                st.launches += 2;
                if (e == cudaSuccess && pass == 0)
                    e = cudaMemcpyAsync(h_dots.data(), dots, sizeof(double2) * (m + 1) * T, cudaMemcpyDeviceToHost, s);
            }
            if (e == cudaSuccess) e = cudaMemcpyAsync(h_norm.data(), dnorm, sizeof(double) * T, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            return e;
        };
        // |w|^2 of every timeslice into h_norm (the inner-product kernel with w as its one basis row)
        auto norm_w = [&]() -> cudaError_t {
            cudaError_t e = cudaMemsetAsync(dots, 0, sizeof(double2) * T, s);
            if (e == cudaSuccess) {
                dots_kernel<<<dim3(blocks_dot, T), LAP_THREADS, 0, s>>>(w, K, w, K, K, 1, dots, 1);
                e = cudaGetLastError();
                st.launches++;
            }
            std::vector<double> tmp(2 * (size_t)T);
            if (e == cudaSuccess) e = cudaMemcpyAsync(tmp.data(), dots, sizeof(double2) * T, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            for (int t = 0; t < T; t++) h_norm[t] = tmp[2 * t];
            return e;
        };
        // the same two passes for the steps without host synchronisation: the
        // first pass's coefficient of basis vector j becomes alpha[t][j], |w|
        // of the result beta[t][j], 1/|w| the scale of basis vector j + 1
        // (dscale), and a step that meets an invariant subspace is noted in dbrk
        auto orthogonalise_dev = [&](int j) -> cudaError_t {
            const unsigned bt = (unsigned)((T + 127) / 128);
            cudaError_t e = cudaSuccess;
            for (int pass = 0; pass < 2 && e == cudaSuccess; pass++) {
                e = cudaMemsetAsync(dots, 0, sizeof(double2) * (m + 1) * T, s);
                if (e == cudaSuccess && pass == 1) e = cudaMemsetAsync(dnorm, 0, sizeof(double) * T, s);
                if (e != cudaSuccess) break;
                dots_kernel<<<dim3(blocks_dot, T), LAP_THREADS, 0, s>>>(basis, ts_b, w, K, K, j + 1, dots, m + 1);
                update_kernel<<<dim3(blocks_upd, T), LAP_THREADS, sizeof(float2) * (j + 1), s>>>(
                    basis, ts_b, w, K, K, j + 1, dots, m + 1, pass == 1 ? dnorm : nullptr);
                if (pass == 0) take_alpha_kernel<<<bt, 128, 0, s>>>(dots, m + 1, j, dalpha, m, T);
                e = cudaGetLastError();
                st.launches += pass == 0 ? 3 : 2;
            }
            if (e == cudaSuccess) {
                take_beta_kernel<<<bt, 128, 0, s>>>(dnorm, dalpha, j, m, T, j + 1 < m ? 1 : 0, dbeta, dscale, dbrk);
                e = cudaGetLastError();
                st.launches++;
            }
            return e;
        };
        // basis vector j = w * dscale (the scales already on the device)
        auto store_dev = [&](int j) -> cudaError_t {
            scale_kernel<<<dim3(blocks_e, T), LAP_THREADS, 0, s>>>(w, K, basis + (long long)j * K, ts_b, K, dscale,
                                                                   d > 0 ? vin : nullptr);
            st.launches++;
            return cudaGetLastError();
        };
        // basis vector j = w * h_scale
        auto store = [&](int j) -> cudaError_t {
            cudaError_t e = cudaMemcpyAsync(dscale, h_scale.data(), sizeof(double) * T, cudaMemcpyHostToDevice, s);
            return e == cudaSuccess ? store_dev(j) : e;
        };

        // the links in the solver's layout; two rows suffice when they are SU(3)
        {
            int *dflag = (int *)(ws + lay.dflag), h_flag = 0;
            LCK(cudaMemsetAsync(dflag, 0, sizeof(int), s));
            const dim3 grid((unsigned)((V + LAP_THREADS - 1) / LAP_THREADS), T);
            if (pairs)
                links_soa_kernel<true><<<grid, LAP_THREADS, 0, s>>>((const float2 *)U, Ud, (unsigned)V, dflag);
            else
                links_soa_kernel<false><<<grid, LAP_THREADS, 0, s>>>((const float2 *)U, Ud, (unsigned)V, dflag);
            LCK(cudaGetLastError());
            st.launches++;
            LCK(cudaMemcpyAsync(&h_flag, dflag, sizeof(int), cudaMemcpyDeviceToHost, s));
            LCK(cudaStreamSynchronize(s));
            r12 = want_r12 && h_flag == 0;
            st.links_two_rows = r12 ? 1 : 0;
        }
        // capture the filter once (on a stream of its own: the caller's may be
        // the legacy default stream, which cannot capture)
        if (d > 0 && n_filter > 1) {
            LCK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
            LCK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
            const cudaError_t e1 = filter_launches(cap);
            const cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
            LCK(e1);
            LCK(e2);
            LCK(cudaGraphInstantiate(&filter, graph, 0));
        }
        // The Krylov steps.  First without host synchronisation: the
        // coefficients alpha, beta and the next vector's scale stay on the
        // device, and come back once after the last step.  If a timeslice met
        // an invariant subspace on the way, the steps run again from the same
        // start vectors (every launch is deterministic, so they repeat up to
        // that step) with the host reading the coefficients after every step
        // and giving the timeslices concerned a fresh vector.
        for (int attempt = 0; attempt < 2; attempt++) {
            const bool host_steps = attempt == 1;
            // start vectors: seeded pattern, normalised
            LCK(laph::launch_fill_pattern(w, K * T, prm->seed ? prm->seed : 12345u, s));
            st.launches++;
            LCK(norm_w());
            for (int t = 0; t < T; t++) h_scale[t] = 1.0 / std::sqrt(std::max(h_norm[t], 1e-300));
            LCK(store(0));
            if (stats && attempt == 0) LCK(cudaEventRecord(ev[1], s));
            if (!host_steps) {
                LCK(cudaMemsetAsync(dbrk, 0x7f, sizeof(int), s));   // 0x7f7f7f7f: no step
                for (int j = 0; j < m; j++) {
                    if (stats) LCK(cudaEventRecord(step_ev[3 * (size_t)j], s));
                    LCK(apply(basis + (long long)j * K));
                    if (stats) LCK(cudaEventRecord(step_ev[3 * (size_t)j + 1], s));
                    LCK(orthogonalise_dev(j));
                    if (stats) LCK(cudaEventRecord(step_ev[3 * (size_t)j + 2], s));
                    if (j + 1 < m) LCK(store_dev(j + 1));
                }
                if (stats) LCK(cudaEventRecord(ev[5], s));
                int h_brk = 0;
                LCK(cudaMemcpyAsync(alpha.data(), dalpha, sizeof(double) * T * m, cudaMemcpyDeviceToHost, s));
                LCK(cudaMemcpyAsync(beta.data(), dbeta, sizeof(double) * T * m, cudaMemcpyDeviceToHost, s));
                LCK(cudaMemcpyAsync(&h_brk, dbrk, sizeof(int), cudaMemcpyDeviceToHost, s));
                LCK(cudaStreamSynchronize(s));
                if (stats)
                    for (int j = 0; j < m; j++) {
                        float a = 0.f, o = 0.f;
                        LCK(cudaEventElapsedTime(&a, step_ev[3 * (size_t)j], step_ev[3 * (size_t)j + 1]));
                        LCK(cudaEventElapsedTime(&o, step_ev[3 * (size_t)j + 1], step_ev[3 * (size_t)j + 2]));
                        st.apply_ms += a;
                        st.orth_ms += o;
                    }
                if (h_brk >= m) break;
                st.host_steps = 1;
                continue;
            }
            for (int j = 0; j < m; j++) {
                if (stats) LCK(cudaEventRecord(ev[2], s));
                LCK(apply(basis + (long long)j * K));
                if (stats) LCK(cudaEventRecord(ev[3], s));
                LCK(orthogonalise(j + 1));
                if (stats) {
                    float a = 0.f, o = 0.f;
                    LCK(cudaEventRecord(ev[4], s));
                    LCK(cudaEventSynchronize(ev[4]));
                    LCK(cudaEventElapsedTime(&a, ev[2], ev[3]));
                    LCK(cudaEventElapsedTime(&o, ev[3], ev[4]));
                    st.apply_ms += a;
                    st.orth_ms += o;
                }
                bool broke = false;
                for (int t = 0; t < T; t++) {
                    const double a = h_dots[2 * ((size_t)t * (m + 1) + j)], b = std::sqrt(std::max(h_norm[t], 0.0));
                    alpha[(size_t)t * m + j] = a;
                    beta[(size_t)t * m + j] = b;
                    h_scale[t] = b > 1e-30 ? 1.0 / b : 0.0;
                    if (b < 1e-6 * std::max(1.0, std::fabs(a))) broke = true;
                }
                if (j + 1 == m) break;
                if (broke) {
                    // an invariant subspace: the timeslices concerned continue from a
                    // fresh vector orthogonal to their basis, with a zero coupling
                    LCK(laph::launch_fill_pattern(ya, K * T, 777u + (unsigned)j, s));
                    st.launches++;
                    for (int t = 0; t < T; t++) {
                        const double a = alpha[(size_t)t * m + j];
                        if (beta[(size_t)t * m + j] < 1e-6 * std::max(1.0, std::fabs(a))) {
                            LCK(cudaMemcpyAsync(w + (long long)t * K, ya + (long long)t * K, sizeof(float2) * K,
                                                cudaMemcpyDeviceToDevice, s));
                            beta[(size_t)t * m + j] = 0.0;
                        }
                    }
                    const std::vector<double> keep = h_dots;
                    LCK(orthogonalise(j + 1));
                    h_dots = keep;
                    for (int t = 0; t < T; t++) h_scale[t] = 1.0 / std::sqrt(std::max(h_norm[t], 1e-300));
                }
                LCK(store(j + 1));
            }
            if (stats) LCK(cudaEventRecord(ev[5], s));
        }
        // Ritz pairs of the tridiagonal matrices; the wanted end: the smallest
        // eigenvalues of -Delta, the largest of the filter (times (-1)^d: T_d
        // grows with sign (-1)^d below the damped interval)
        {
            // the timeslices' tridiagonal problems are independent: host threads share them
            const double sgn = (d % 2) ? -1.0 : 1.0;
            const int n_thr = (int)std::max(1u, std::min<unsigned>((unsigned)T, std::min(32u, std::thread::hardware_concurrency())));
            std::vector<int> failed(n_thr, 0);
            auto work = [&](int id) {
                std::vector<double> dd(m), ee(m), z((size_t)m * m);
                for (int t = id; t < T; t += n_thr) {
                    for (int i = 0; i < m; i++) dd[i] = alpha[(size_t)t * m + i];
                    for (int i = 0; i + 1 < m; i++) ee[i] = beta[(size_t)t * m + i];
                    if (laph::tridiag_eigen(m, dd.data(), ee.data(), z.data()) != 0) {
                        failed[id] = 1;
                        return;
                    }
                    for (int r = 0; r < nr; r++) {
                        const int k = (d > 0 && sgn > 0) ? m - 1 - r : r;
                        for (int i = 0; i < m; i++) h_S[((size_t)t * m + i) * nr + r] = z[(size_t)i * m + k];
                    }
                }
            };
            std::vector<std::thread> pool;
            for (int id = 1; id < n_thr; id++) pool.emplace_back(work, id);
            work(0);
            for (auto &th : pool) th.join();
            for (int f : failed)
                if (f) {
                    rc = LAPH_ERR_ARG;
                    goto done;
                }
        }
        LCK(cudaMemcpyAsync(dS, h_S.data(), sizeof(double) * T * m * nr, cudaMemcpyHostToDevice, s));
        ritz_kernel<<<dim3(blocks_e, T, (nr + RT - 1) / RT), LAP_THREADS, 0, s>>>(basis, ts_b, K, m, dS, nr, X,
                                                                                   K * nr);
        LCK(cudaGetLastError());
        // Rayleigh quotients and residuals with -Delta (Y reuses the basis)
        LCK(launch_lap_soa(Ud, X, nullptr, Y, L, T, nr, K * nr, 0, K * nr, 1.f, 0.f, 0.f, s, r12, pairs));
        LCK(cudaMemsetAsync(dred, 0, sizeof(double) * 2 * T * nr, s));
        st.launches += 5;   // Ritz vectors, -Delta on them, two Rayleigh passes, gather
        {
            const unsigned rb = std::min<unsigned>(blocks_e, 64u);
            rayleigh_kernel<<<dim3(rb, T, nr), LAP_THREADS, 0, s>>>(X, Y, K * nr, K, 0, nullptr, nr, dred);
            LCK(cudaGetLastError());
            LCK(cudaMemcpyAsync(h_red.data(), dred, sizeof(double) * 2 * T * nr, cudaMemcpyDeviceToHost, s));
            LCK(cudaStreamSynchronize(s));
            std::vector<double> lam((size_t)T * nr), xx((size_t)T * nr);
            for (size_t i = 0; i < (size_t)T * nr; i++) {
                xx[i] = h_red[2 * i + 1];
                lam[i] = h_red[2 * i] / std::max(xx[i], 1e-300);
            }
            LCK(cudaMemcpyAsync(dlam, lam.data(), sizeof(double) * T * nr, cudaMemcpyHostToDevice, s));
            LCK(cudaMemsetAsync(dred, 0, sizeof(double) * 2 * T * nr, s));
            rayleigh_kernel<<<dim3(rb, T, nr), LAP_THREADS, 0, s>>>(X, Y, K * nr, K, 1, dlam, nr, dred);
            LCK(cudaGetLastError());
            LCK(cudaMemcpyAsync(h_red.data(), dred, sizeof(double) * 2 * T * nr, cudaMemcpyDeviceToHost, s));
            LCK(cudaStreamSynchronize(s));
            // ascending eigenvalues per timeslice; the vectors leave with unit norm
            std::vector<int> perm((size_t)T * nr);
            std::vector<double> inv_norm((size_t)T * nr);
            for (int t = 0; t < T; t++) {
                int *pt = perm.data() + (size_t)t * nr;
                for (int r = 0; r < nr; r++) pt[r] = r;
                std::sort(pt, pt + nr, [&](int a, int b) { return lam[(size_t)t * nr + a] < lam[(size_t)t * nr + b]; });
                for (int r = 0; r < nr; r++) {
                    const size_t src = (size_t)t * nr + pt[r];
                    evals[(size_t)t * nr + r] = lam[src];
                    inv_norm[(size_t)t * nr + r] = 1.0 / std::sqrt(std::max(xx[src], 1e-300));
                    if (resid) resid[(size_t)t * nr + r] = std::sqrt(std::max(h_red[2 * src], 0.0) / std::max(xx[src], 1e-300));
                }
            }
            LCK(cudaMemcpyAsync(dperm, perm.data(), sizeof(int) * T * nr, cudaMemcpyHostToDevice, s));
            LCK(cudaMemcpyAsync(dred, inv_norm.data(), sizeof(double) * T * nr, cudaMemcpyHostToDevice, s));
            if (pairs)
                gather_kernel<true><<<dim3(blocks_e, T, nr), LAP_THREADS, 0, s>>>(X, K * nr, dperm, dred, nr,
                                                                                (float2 *)evecs, K * nr, V);
            else
                gather_kernel<false><<<dim3(blocks_e, T, nr), LAP_THREADS, 0, s>>>(X, K * nr, dperm, dred, nr,
                                                                                 (float2 *)evecs, K * nr, V);
            LCK(cudaGetLastError());
            if (stats) {
                float tot = 0.f, setup = 0.f, ritz = 0.f;
                LCK(cudaEventRecord(ev[6], s));
                LCK(cudaEventSynchronize(ev[6]));
                LCK(cudaEventElapsedTime(&tot, ev[0], ev[6]));
                LCK(cudaEventElapsedTime(&setup, ev[0], ev[1]));
                LCK(cudaEventElapsedTime(&ritz, ev[5], ev[6]));
                st.total_ms = tot;
                st.setup_ms = setup;
                st.ritz_ms = ritz;
                *stats = st;
            }
            LCK(cudaStreamSynchronize(s));
        }
    }
done:
    for (auto &e : ev)
        if (e) cudaEventDestroy(e);
    for (auto &e : step_ev)
        if (e) cudaEventDestroy(e);
    if (filter) cudaGraphExecDestroy(filter);
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
    if (owned) cudaFreeAsync(owned, s);
    cudaStreamSynchronize(s);
    return rc;
}

}  // extern "C"
