/*
 * FP64 CPU oracle for the LapH meson/baryon block contraction.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into a small shared
 * library that is loaded by the tests, by the smoke check and by the
 * CPU-baseline leg of the benchmark.  The product (the CUDA library) never
 * links, loads or calls it, and it shares no code, header, table or helper
 * with the CUDA path.
 *
 * What it computes (paper: section "Innovations", subsection "QUDA": the
 * LapH eigenvectors are used to form quark-antiquark doublets and
 * three-quark triplets for the meson and baryon sources and sinks; LapH
 * smearing itself is introduced in section "Current state-of-the-art").
 * For one timeslice with N complex colour vectors phi_i^a(x) on an L^3
 * spatial lattice and a list of integer momenta n_p (p = 2 pi n_p / L):
 *
 *   ph_p(x)      = exp(-2 pi i ((n_p . x) mod L) / L)
 *   B[p][i,j,k]  = sum_x ph_p(x) sum_{a,b,c} eps_abc phi_i^a(x) phi_j^b(x) phi_k^c(x)
 *   M[p][i][j]   = sum_x ph_p(x) sum_a conj(phi_i^a(x)) phi_j^a(x)
 *
 * Readings taken where the paper is silent (each is listed in the design
 * notes): site index x = x0 + L*x1 + L*L*x2 with x0 fastest, origin 0,
 * periodic; no 1/V normalisation; no conjugation in B; M conjugates its
 * first index; packed baryon storage keeps i<j<k only, at the colex index
 * C(k,3) + C(j,2) + i.
 *
 * Everything is done in double precision with plain loops in the order of
 * the definition: for each output element, loop over sites, form the
 * epsilon sum (or colour dot product) at that site, multiply by the phase,
 * accumulate.  The only hoisting is that the site term, which does not
 * depend on p, is formed once and multiplied by each momentum's phase.
 * OpenMP distributes independent output elements over threads; every
 * element is summed by one thread in site order, so results do not depend
 * on the thread count.
 *
 * Data layout: complex numbers are (re, im) pairs of doubles.
 *   phi  [N][V][3]      (vector, site, colour)
 *   mom  [P][3]         int32 (n_x, n_y, n_z)
 *   B    [P][C(N,3)]    packed
 *   M    [P][N][N]
 *
 * General fields (three different sets of N colour vectors phi, psi, chi,
 * e.g. stochastic-LapH quark sinks; same paper passage):
 *
 *   B3[p][i][j][k] = sum_x ph_p(x) sum_{a,b,c} eps_abc phi_i^a(x) psi_j^b(x) chi_k^c(x)   (dense, no symmetry)
 *   M2[p][i][j]    = sum_x ph_p(x) sum_a conj(phi_i^a(x)) psi_j^a(x)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double re, im;
} cplx;

static cplx cmul(cplx a, cplx b)
{
    cplx r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
    return r;
}

static cplx cconj(cplx a)
{
    cplx r = {a.re, -a.im};
    return r;
}

static int64_t binom2(int64_t n) { return n * (n - 1) / 2; }
static int64_t binom3(int64_t n) { return n * (n - 1) * (n - 2) / 6; }

/* Levi-Civita symbol eps_abc as its six non-zero entries. */
static const int EPS_PERM[6][3] = {{0, 1, 2}, {1, 2, 0}, {2, 0, 1}, {0, 2, 1}, {2, 1, 0}, {1, 0, 2}};
static const double EPS_SIGN[6] = {+1.0, +1.0, +1.0, -1.0, -1.0, -1.0};

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ph_p(x) = exp(-2 pi i r / L) with r = (n . x) mod L taken in [0, L). */
static cplx phase_at(int L, const int32_t n[3], int64_t x)
{
    int64_t x0 = x % L, x1 = (x / L) % L, x2 = x / ((int64_t)L * L);
    int64_t r = ((int64_t)n[0] * x0 + (int64_t)n[1] * x1 + (int64_t)n[2] * x2) % L;
    if (r < 0) r += L;
    double ang = -2.0 * M_PI * (double)r / (double)L;
    cplx z = {cos(ang), sin(ang)};
    return z;
}

/* out[P][V] complex: the momentum phase of every site. */
void oracle_phase_table(int L, const int32_t *mom, int P, double *out)
{
    int64_t V = (int64_t)L * L * L;
    for (int p = 0; p < P; p++)
        for (int64_t x = 0; x < V; x++) {
            cplx z = phase_at(L, &mom[3 * p], x);
            out[2 * (p * V + x)] = z.re;
            out[2 * (p * V + x) + 1] = z.im;
        }
}

/* Site-major copy of the phases, phT[x][p], so that the p loop is contiguous. */
static cplx *phase_site_major(int L, const int32_t *mom, int P)
{
    int64_t V = (int64_t)L * L * L;
    cplx *phT = (cplx *)malloc(sizeof(cplx) * (size_t)(V * P));
    if (!phT) return NULL;
    for (int64_t x = 0; x < V; x++)
        for (int p = 0; p < P; p++) phT[x * P + p] = phase_at(L, &mom[3 * p], x);
    return phT;
}

static cplx phi_at(const double *phi, int64_t V, int i, int64_t x, int a)
{
    const double *q = phi + 2 * ((i * V + x) * 3 + a);
    cplx z = {q[0], q[1]};
    return z;
}

/* eps_abc phi_i^a(x) phi_j^b(x) phi_k^c(x), summed over the six permutations. */
static cplx eps_site(const double *phi, int64_t V, int i, int j, int k, int64_t x)
{
    cplx s = {0.0, 0.0};
    for (int q = 0; q < 6; q++) {
        cplx t = cmul(cmul(phi_at(phi, V, i, x, EPS_PERM[q][0]), phi_at(phi, V, j, x, EPS_PERM[q][1])),
                      phi_at(phi, V, k, x, EPS_PERM[q][2]));
        s.re += EPS_SIGN[q] * t.re;
        s.im += EPS_SIGN[q] * t.im;
    }
    return s;
}

/*
 * Baryon block for an arbitrary list of index triples (any order, repeats
 * allowed): out[n][P] complex = B[p][ijk[n][0], ijk[n][1], ijk[n][2]].
 * Returns 0, or -1 on allocation failure / bad index.
 */
int oracle_baryon_triples(const double *phi, int L, int N, const int32_t *mom, int P, int64_t n_trip,
                          const int32_t *ijk, double *out)
{
    int64_t V = (int64_t)L * L * L;
    for (int64_t t = 0; t < 3 * n_trip; t++)
        if (ijk[t] < 0 || ijk[t] >= N) return -1;
    cplx *phT = phase_site_major(L, mom, P);
    if (!phT) return -1;
    int failed = 0;
#pragma omp parallel
    {
        cplx *acc = (cplx *)malloc(sizeof(cplx) * (size_t)P);
        if (!acc) {
#pragma omp atomic write
            failed = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t t = 0; t < n_trip; t++) {
            if (!acc) continue;
            int i = ijk[3 * t], j = ijk[3 * t + 1], k = ijk[3 * t + 2];
            for (int p = 0; p < P; p++) acc[p].re = acc[p].im = 0.0;
            for (int64_t x = 0; x < V; x++) {
                cplx e = eps_site(phi, V, i, j, k, x);
                const cplx *ph = phT + x * P;
                for (int p = 0; p < P; p++) {
                    cplx u = cmul(ph[p], e);
                    acc[p].re += u.re;
                    acc[p].im += u.im;
                }
            }
            for (int p = 0; p < P; p++) {
                out[2 * (t * P + p)] = acc[p].re;
                out[2 * (t * P + p) + 1] = acc[p].im;
            }
        }
        free(acc);
    }
    free(phT);
    return failed ? -1 : 0;
}

/*
 * Packed baryon blocks: out[P][C(N,3)] complex, element (i<j<k) at the colex
 * index C(k,3) + C(j,2) + i.
 */
int oracle_baryon_blocks(const double *phi, int L, int N, const int32_t *mom, int P, double *out)
{
    int64_t T3 = binom3(N);
    if (T3 == 0) return 0;
    int32_t *ijk = (int32_t *)malloc(sizeof(int32_t) * (size_t)(3 * T3));
    double *tmp = (double *)malloc(sizeof(double) * (size_t)(2 * T3 * P));
    if (!ijk || !tmp) {
        free(ijk);
        free(tmp);
        return -1;
    }
    for (int k = 2; k < N; k++)
        for (int j = 1; j < k; j++)
            for (int i = 0; i < j; i++) {
                int64_t idx = binom3(k) + binom2(j) + i;
                ijk[3 * idx] = i;
                ijk[3 * idx + 1] = j;
                ijk[3 * idx + 2] = k;
            }
    int rc = oracle_baryon_triples(phi, L, N, mom, P, T3, ijk, tmp);
    if (rc == 0)
        for (int64_t idx = 0; idx < T3; idx++)
            for (int p = 0; p < P; p++) {
                out[2 * (p * T3 + idx)] = tmp[2 * (idx * P + p)];
                out[2 * (p * T3 + idx) + 1] = tmp[2 * (idx * P + p) + 1];
            }
    free(ijk);
    free(tmp);
    return rc;
}

/* Meson blocks: out[P][N][N] complex, M[p][i][j] = sum_x ph_p(x) sum_a conj(phi_i^a) phi_j^a. */
int oracle_meson_blocks(const double *phi, int L, int N, const int32_t *mom, int P, double *out)
{
    int64_t V = (int64_t)L * L * L;
    cplx *phT = phase_site_major(L, mom, P);
    if (!phT) return -1;
    int failed = 0;
#pragma omp parallel
    {
        cplx *acc = (cplx *)malloc(sizeof(cplx) * (size_t)P);
        if (!acc) {
#pragma omp atomic write
            failed = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t ij = 0; ij < (int64_t)N * N; ij++) {
            if (!acc) continue;
            int i = (int)(ij / N), j = (int)(ij % N);
            for (int p = 0; p < P; p++) acc[p].re = acc[p].im = 0.0;
            for (int64_t x = 0; x < V; x++) {
                cplx s = {0.0, 0.0};
                for (int a = 0; a < 3; a++) {
                    cplx u = cmul(cconj(phi_at(phi, V, i, x, a)), phi_at(phi, V, j, x, a));
                    s.re += u.re;
                    s.im += u.im;
                }
                const cplx *ph = phT + x * P;
                for (int p = 0; p < P; p++) {
                    cplx u = cmul(ph[p], s);
                    acc[p].re += u.re;
                    acc[p].im += u.im;
                }
            }
            for (int p = 0; p < P; p++) {
                out[2 * ((p * (int64_t)N + i) * N + j)] = acc[p].re;
                out[2 * ((p * (int64_t)N + i) * N + j) + 1] = acc[p].im;
            }
        }
        free(acc);
    }
    free(phT);
    return failed ? -1 : 0;
}

/*
 * Diquarks: out[C(N,2)][V][3] complex, D_q(x)_c = sum_{a,b} eps_cab phi_i^a(x) phi_j^b(x)
 * for the pair q = C(j,2) + i, i < j.
 */
void oracle_diquarks(const double *phi, int L, int N, double *out)
{
    int64_t V = (int64_t)L * L * L;
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = 1; j < N; j++)
        for (int i = 0; i < j; i++) {
            int64_t q = binom2(j) + i;
            for (int64_t x = 0; x < V; x++) {
                cplx d[3] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
                for (int t = 0; t < 6; t++) {
                    /* eps_cab = eps_abc: permutation (c,a,b) of the table entry (a,b,c) */
                    int a = EPS_PERM[t][0], b = EPS_PERM[t][1], c = EPS_PERM[t][2];
                    cplx u = cmul(phi_at(phi, V, i, x, a), phi_at(phi, V, j, x, b));
                    d[c].re += EPS_SIGN[t] * u.re;
                    d[c].im += EPS_SIGN[t] * u.im;
                }
                for (int c = 0; c < 3; c++) {
                    out[2 * ((q * V + x) * 3 + c)] = d[c].re;
                    out[2 * ((q * V + x) * 3 + c) + 1] = d[c].im;
                }
            }
        }
}

/*
 * Dense baryon tensor from the packed form: dense[P][N][N][N] with
 * dense[p][a][b][c] = sign(sort permutation of (a,b,c)) * B[p][sorted], and 0
 * when two indices coincide.  Written straight from the antisymmetry of
 * eps_abc.
 */
void oracle_baryon_dense(const double *packed, int N, int P, double *dense)
{
    int64_t T3 = binom3(N);
    for (int p = 0; p < P; p++)
        for (int a = 0; a < N; a++)
            for (int b = 0; b < N; b++)
                for (int c = 0; c < N; c++) {
                    int64_t o = 2 * (((p * (int64_t)N + a) * N + b) * N + c);
                    int v[3] = {a, b, c};
                    double sign = 1.0;
                    /* bubble sort, counting swaps */
                    for (int s = 0; s < 2; s++)
                        for (int q = 0; q < 2 - s; q++)
                            if (v[q] > v[q + 1]) {
                                int tmp = v[q];
                                v[q] = v[q + 1];
                                v[q + 1] = tmp;
                                sign = -sign;
                            }
                    if (v[0] == v[1] || v[1] == v[2]) {
                        dense[o] = 0.0;
                        dense[o + 1] = 0.0;
                        continue;
                    }
                    int64_t idx = binom3(v[2]) + binom2(v[1]) + v[0];
                    dense[o] = sign * packed[2 * (p * T3 + idx)];
                    dense[o + 1] = sign * packed[2 * (p * T3 + idx) + 1];
                }
}

/* eps_abc f1_i^a(x) f2_j^b(x) f3_k^c(x) for three different fields, summed over the six permutations. */
static cplx eps_site_fields(const double *f1, const double *f2, const double *f3, int64_t V, int i, int j, int k,
                            int64_t x)
{
    cplx s = {0.0, 0.0};
    for (int q = 0; q < 6; q++) {
        cplx t = cmul(cmul(phi_at(f1, V, i, x, EPS_PERM[q][0]), phi_at(f2, V, j, x, EPS_PERM[q][1])),
                      phi_at(f3, V, k, x, EPS_PERM[q][2]));
        s.re += EPS_SIGN[q] * t.re;
        s.im += EPS_SIGN[q] * t.im;
    }
    return s;
}

/*
 * Three-field triplets for a list of index triples: out[n][P] complex =
 * B3[p][ijk[n][0], ijk[n][1], ijk[n][2]] with field f1 = phi at index i,
 * f2 = psi at j, f3 = chi at k.  Returns 0, or -1 on allocation failure /
 * bad index.
 */
int oracle_triplet_triples(const double *f1, const double *f2, const double *f3, int L, int N, const int32_t *mom,
                           int P, int64_t n_trip, const int32_t *ijk, double *out)
{
    int64_t V = (int64_t)L * L * L;
    for (int64_t t = 0; t < 3 * n_trip; t++)
        if (ijk[t] < 0 || ijk[t] >= N) return -1;
    cplx *phT = phase_site_major(L, mom, P);
    if (!phT) return -1;
    int failed = 0;
#pragma omp parallel
    {
        cplx *acc = (cplx *)malloc(sizeof(cplx) * (size_t)P);
        if (!acc) {
#pragma omp atomic write
            failed = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t t = 0; t < n_trip; t++) {
            if (!acc) continue;
            int i = ijk[3 * t], j = ijk[3 * t + 1], k = ijk[3 * t + 2];
            for (int p = 0; p < P; p++) acc[p].re = acc[p].im = 0.0;
            for (int64_t x = 0; x < V; x++) {
                cplx e = eps_site_fields(f1, f2, f3, V, i, j, k, x);
                const cplx *ph = phT + x * P;
                for (int p = 0; p < P; p++) {
                    cplx u = cmul(ph[p], e);
                    acc[p].re += u.re;
                    acc[p].im += u.im;
                }
            }
            for (int p = 0; p < P; p++) {
                out[2 * (t * P + p)] = acc[p].re;
                out[2 * (t * P + p) + 1] = acc[p].im;
            }
        }
        free(acc);
    }
    free(phT);
    return failed ? -1 : 0;
}

/* Dense three-field triplets: out[P][N][N][N] complex, element [p][i][j][k]. */
int oracle_triplet_blocks(const double *f1, const double *f2, const double *f3, int L, int N, const int32_t *mom,
                          int P, double *out)
{
    int64_t n3 = (int64_t)N * N * N;
    if (n3 == 0) return 0;
    int32_t *ijk = (int32_t *)malloc(sizeof(int32_t) * (size_t)(3 * n3));
    double *tmp = (double *)malloc(sizeof(double) * (size_t)(2 * n3 * P));
    if (!ijk || !tmp) {
        free(ijk);
        free(tmp);
        return -1;
    }
    for (int64_t e = 0; e < n3; e++) {
        ijk[3 * e] = (int32_t)(e / ((int64_t)N * N));
        ijk[3 * e + 1] = (int32_t)((e / N) % N);
        ijk[3 * e + 2] = (int32_t)(e % N);
    }
    int rc = oracle_triplet_triples(f1, f2, f3, L, N, mom, P, n3, ijk, tmp);
    if (rc == 0)
        for (int64_t e = 0; e < n3; e++)
            for (int p = 0; p < P; p++) {
                out[2 * (p * n3 + e)] = tmp[2 * (e * P + p)];
                out[2 * (p * n3 + e) + 1] = tmp[2 * (e * P + p) + 1];
            }
    free(ijk);
    free(tmp);
    return rc;
}

/*
 * Projection of one set of colour vectors onto another (paper, section
 * "Innovations", subsection "Eigenvector Projection": inner products of the
 * solution vectors with the LapH eigenvectors), with a momentum phase:
 * out[P][N1][N2] complex, out[p][i][j] = sum_x ph_p(x) sum_a conj(f1_i^a(x)) f2_j^a(x),
 * f1 [N1][V][3], f2 [N2][V][3].  With the single momentum n = 0 this is the
 * plain inner product <f1_i, f2_j>.
 */
int oracle_projection(const double *f1, const double *f2, int L, int N1, int N2, const int32_t *mom, int P,
                      double *out)
{
    int64_t V = (int64_t)L * L * L;
    cplx *phT = phase_site_major(L, mom, P);
    if (!phT) return -1;
    int failed = 0;
#pragma omp parallel
    {
        cplx *acc = (cplx *)malloc(sizeof(cplx) * (size_t)P);
        if (!acc) {
#pragma omp atomic write
            failed = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t ij = 0; ij < (int64_t)N1 * N2; ij++) {
            if (!acc) continue;
            int i = (int)(ij / N2), j = (int)(ij % N2);
            for (int p = 0; p < P; p++) acc[p].re = acc[p].im = 0.0;
            for (int64_t x = 0; x < V; x++) {
                cplx s = {0.0, 0.0};
                for (int a = 0; a < 3; a++) {
                    cplx u = cmul(cconj(phi_at(f1, V, i, x, a)), phi_at(f2, V, j, x, a));
                    s.re += u.re;
                    s.im += u.im;
                }
                const cplx *ph = phT + x * P;
                for (int p = 0; p < P; p++) {
                    cplx u = cmul(ph[p], s);
                    acc[p].re += u.re;
                    acc[p].im += u.im;
                }
            }
            for (int p = 0; p < P; p++) {
                int64_t o = 2 * ((p * (int64_t)N1 + i) * N2 + j);   /* [p][i][j] */
                out[o] = acc[p].re;
                out[o + 1] = acc[p].im;
            }
        }
        free(acc);
    }
    free(phT);
    return failed ? -1 : 0;
}

/* Two-field doublets: out[P][N][N] complex, M2[p][i][j] = sum_x ph_p(x) sum_a conj(f1_i^a) f2_j^a
 * (the projection of N vectors onto N vectors). */
int oracle_doublet_blocks(const double *f1, const double *f2, int L, int N, const int32_t *mom, int P, double *out)
{
    return oracle_projection(f1, f2, L, N, N, mom, P, out);
}

/*
 * The 3-d gauge-covariant Laplacian of one timeslice, whose lowest
 * eigenvectors are the LapH vectors (paper, section "Innovations",
 * subsection "Scalable Lanczos Eigensolver"):
 *
 *   (-Delta f)(x) = sum_mu [ 2 f(x) - U_mu(x) f(x + mu) - U_mu(x - mu)^dagger f(x - mu) ]
 *
 * over the three spatial directions mu, periodic.  U [3][V][3][3] complex
 * (row-major colour matrices), f and out [nvec][V][3] complex.
 */
void oracle_laplacian(const double *U, const double *f, int L, int nvec, double *out)
{
    int64_t V = (int64_t)L * L * L;
#pragma omp parallel for schedule(static)
    for (int64_t nx = 0; nx < (int64_t)nvec * V; nx++) {
        int64_t n = nx / V, x = nx % V;
        int64_t c[3] = {x % L, (x / L) % L, x / ((int64_t)L * L)};
        const int64_t stride[3] = {1, L, (int64_t)L * L};
        cplx acc[3];
        for (int a = 0; a < 3; a++) {
            cplx v = phi_at(f, V, (int)n, x, a);
            acc[a].re = 6.0 * v.re;
            acc[a].im = 6.0 * v.im;
        }
        for (int mu = 0; mu < 3; mu++) {
            int64_t up = x + (c[mu] == L - 1 ? -(int64_t)(L - 1) * stride[mu] : stride[mu]);
            int64_t dn = x - (c[mu] == 0 ? -(int64_t)(L - 1) * stride[mu] : stride[mu]);
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) {
                    /* U_mu(x)_{ab} f_b(x + mu) */
                    const double *u = U + 2 * (((mu * V + x) * 3 + a) * 3 + b);
                    cplx uf = cmul((cplx){u[0], u[1]}, phi_at(f, V, (int)n, up, b));
                    /* (U_mu(x - mu)^dagger)_{ab} f_b(x - mu) = conj(U_mu(x - mu)_{ba}) f_b(x - mu) */
                    const double *w = U + 2 * (((mu * V + dn) * 3 + b) * 3 + a);
                    cplx wf = cmul(cconj((cplx){w[0], w[1]}), phi_at(f, V, (int)n, dn, b));
                    acc[a].re -= uf.re + wf.re;
                    acc[a].im -= uf.im + wf.im;
                }
        }
        for (int a = 0; a < 3; a++) {
            out[2 * ((n * V + x) * 3 + a)] = acc[a].re;
            out[2 * ((n * V + x) * 3 + a) + 1] = acc[a].im;
        }
    }
}
