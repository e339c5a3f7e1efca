/*
 * FP64 CPU oracle for CNN variational Monte Carlo on the spin-1/2 J1-J2
 * Heisenberg model (arXiv:2108.13830).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code with the CUDA library.
 *
 * Every routine is the plain definition, in double precision, with loops in
 * the order the definition reads:
 *   - Hamiltonian, Eq. 3 (Sec. 2.1): H = J1/4 sum_<ij> sigma_i.sigma_j
 *     + J2/4 sum_<<ij>> sigma_i.sigma_j on an L x L torus.  Bonds are listed
 *     per site as in Sec. 3.1 / Fig. 2c: right and below neighbour for J1,
 *     the two lower diagonals (down-right, down-left) for J2.
 *   - Matrix elements from the Pauli matrices, Eq. 2: diagonal
 *     (J/4) s_i s_j, and J/2 between configurations that differ by the
 *     exchange of an antiparallel pair.
 *   - Local energy E_s = sum_S' H_S'S w(S')/w(S), Eq. 4-5, evaluated with the
 *     full signs of w (no shortcut for the Marshall factor).
 *   - CNN amplitude: 3x3 circular-padded convolutions, SiLU on all layers
 *     but the last, product pooling of the last layer:
 *     log|w_CNN| = sum_{c,p} log|z_{c,p}|, sign = prod sgn z_{c,p}, times the
 *     Marshall-Peierls sign (-1)^{M_A} of Eq. 9 (M_A = number of up spins on
 *     the sublattice x + y even).
 *   - Log-derivatives O_k = (1/w) dw/da_k, Eq. 5, by hand-written reverse
 *     mode.
 *   - SR: <O>, <E>, G = <O E> - <E><O> (Eq. 5), the covariance product
 *     M v = (1/m) O^T (O v) - <O> (<O> . v) (Eq. 7 and the construction of
 *     M in Sec. 3.2.2) plus a diagonal shift, and plain conjugate gradient
 *     on (M + shift I) x = G.
 *
 * Parameter layout (flat vector): for l = 0..D, W_l[c_out][c_in][ky][kx]
 * then b_l[c_out]; c_in = 1 for l = 0, C otherwise; c_out = C.
 * Convolution: z[co][y][x] = b[co] + sum_{ci,ky,kx} W[co][ci][ky][kx]
 *              * a[ci][(y+ky-1) mod L][(x+kx-1) mod L].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int64_t orc_num_params(int C, int D) { return (int64_t)(10 * C) + (int64_t)D * (9 * C * C + C); }

static double silu(double z) { return z / (1.0 + exp(-z)); }
static double sigmoid(double z) { return 1.0 / (1.0 + exp(-z)); }

/* Offset of W_l in the flat vector. */
static int64_t w_offset(int C, int l)
{
    if (l == 0) return 0;
    return (int64_t)(10 * C) + (int64_t)(l - 1) * (9 * C * C + C);
}

/* All pre-activations z_l[C][N], l = 0..D, into z ((D+1)*C*N doubles). */
static void cnn_forward(int L, int C, int D, const double *theta, const int8_t *s, double *z)
{
    const int N = L * L;
    double *a = (double *)malloc(sizeof(double) * (size_t)C * N);
    /* site of tap (ky, kx) around each site, t = 3 ky + kx, mod L */
    int *nbr = (int *)malloc(sizeof(int) * 9 * (size_t)N);
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x)
            for (int ky = 0; ky < 3; ++ky)
                for (int kx = 0; kx < 3; ++kx)
                    nbr[9 * (y * L + x) + 3 * ky + kx] = ((y + ky - 1 + L) % L) * L + (x + kx - 1 + L) % L;
    for (int l = 0; l <= D; ++l) {
        const int cin = (l == 0) ? 1 : C;
        const double *W = theta + w_offset(C, l);
        const double *b = W + 9 * C * cin;
        double *zl = z + (size_t)l * C * N;
        if (l > 0) {
            const double *zp = z + (size_t)(l - 1) * C * N;
            for (int i = 0; i < C * N; ++i) a[i] = silu(zp[i]);
        }
        for (int co = 0; co < C; ++co)
            for (int y = 0; y < L; ++y)
                for (int x = 0; x < L; ++x) {
                    const int *nb = nbr + 9 * (y * L + x);
                    double acc = b[co];
                    for (int ci = 0; ci < cin; ++ci) {
                        const double *Wc = W + (co * cin + ci) * 9;
                        const double *ac = a + (size_t)ci * N;
                        for (int t = 0; t < 9; ++t) {
                            const double in = (l == 0) ? (double)s[nb[t]] : ac[nb[t]];
                            acc += Wc[t] * in;
                        }
                    }
                    zl[co * N + y * L + x] = acc;
                }
    }
    free(nbr);
    free(a);
}

/* (-1)^{M_A}, M_A = number of up spins on the sublattice x + y even (Eq. 9). */
static int marshall_sign(int L, const int8_t *s)
{
    int ma = 0;
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x)
            if (((x + y) & 1) == 0 && s[y * L + x] == 1) ++ma;
    return (ma & 1) ? -1 : 1;
}

/* Product pooling of the last layer: log|w| and sign (0 when some z == 0). */
static void pool(int N, int C, const double *zD, double *logabs, int *sign)
{
    double acc = 0.0;
    int sg = 1;
    for (int i = 0; i < C * N; ++i) {
        if (zD[i] == 0.0) { *logabs = -INFINITY; *sign = 0; return; }
        acc += log(fabs(zD[i]));
        if (zD[i] < 0.0) sg = -sg;
    }
    *logabs = acc;
    *sign = sg;
}

void orc_forward_z(int L, int C, int D, const double *theta, const int8_t *s, double *z)
{
    cnn_forward(L, C, D, theta, s, z);
}

void orc_logpsi(int L, int C, int D, const double *theta, int marshall,
                const int8_t *s, double *logabs, int *sign)
{
    const int N = L * L;
    double *z = (double *)malloc(sizeof(double) * (size_t)(D + 1) * C * N);
    cnn_forward(L, C, D, theta, s, z);
    pool(N, C, z + (size_t)D * C * N, logabs, sign);
    if (marshall) *sign *= marshall_sign(L, s);
    free(z);
}

/* ---- local energy, generic in the wavefunction ------------------------- */

typedef void (*wf_fn)(const void *ctx, const int8_t *s, double *logabs, int *sign);

typedef struct { int L, C, D, marshall; const double *theta; } cnn_ctx;

static void cnn_wf(const void *ctx, const int8_t *s, double *logabs, int *sign)
{
    const cnn_ctx *c = (const cnn_ctx *)ctx;
    orc_logpsi(c->L, c->C, c->D, c->theta, c->marshall, s, logabs, sign);
}

/* Lookup-table wavefunction for L = 4: index = sum_i [s_i = +1] 2^i. */
typedef struct { int L; const double *table; } table_ctx;

static void table_wf(const void *ctx, const int8_t *s, double *logabs, int *sign)
{
    const table_ctx *t = (const table_ctx *)ctx;
    const int N = t->L * t->L;
    uint32_t idx = 0;
    for (int i = 0; i < N; ++i)
        if (s[i] == 1) idx |= 1u << i;
    double v = t->table[idx];
    *logabs = (v == 0.0) ? -INFINITY : log(fabs(v));
    *sign = (v > 0.0) - (v < 0.0);
}

/* Bond (i, j) of type t at site (y, x): t = 0 right, 1 down (J1);
 * t = 2 down-right, 3 down-left (J2).  Fig. 2c / Sec. 3.1. */
static int bond_partner(int L, int y, int x, int t)
{
    static const int dy[4] = {0, 1, 1, 1}, dx[4] = {1, 0, 1, -1};
    int yy = (y + dy[t]) % L, xx = (x + dx[t] + L) % L;
    return yy * L + xx;
}

static double local_energy(int L, double J1, double J2, const int8_t *s,
                           wf_fn wf, const void *ctx, int *n_nbr)
{
    const int N = L * L;
    int8_t *sp = (int8_t *)malloc((size_t)N);
    double la; int sa;
    wf(ctx, s, &la, &sa);
    double e = 0.0;
    int nn = 0;
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x)
            for (int t = 0; t < 4; ++t) {
                const int i = y * L + x, j = bond_partner(L, y, x, t);
                const double J = (t < 2) ? J1 : J2;
                if (s[i] == s[j]) { e += J / 4.0; continue; }
                e -= J / 4.0;
                memcpy(sp, s, (size_t)N);
                sp[i] = s[j];
                sp[j] = s[i];
                double lb; int sb;
                wf(ctx, sp, &lb, &sb);
                e += (J / 2.0) * ((double)sb / (double)sa) * exp(lb - la);
                ++nn;
            }
    free(sp);
    if (n_nbr) *n_nbr = nn;
    return e;
}

double orc_local_energy_cnn(int L, double J1, double J2, int C, int D, const double *theta,
                            int marshall, const int8_t *s, int *n_nbr)
{
    cnn_ctx c = {L, C, D, marshall, theta};
    return local_energy(L, J1, J2, s, cnn_wf, &c, n_nbr);
}

double orc_local_energy_table(int L, double J1, double J2, const double *table, const int8_t *s)
{
    table_ctx t = {L, table};
    return local_energy(L, J1, J2, s, table_wf, &t, NULL);
}

/* Batched forms (OpenMP over samples; used for timing and large tests). */
void orc_logpsi_batch(int L, int C, int D, const double *theta, int marshall,
                      const int8_t *s, int64_t B, double *logabs, int *sign, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t b = 0; b < B; ++b)
        orc_logpsi(L, C, D, theta, marshall, s + b * L * L, logabs + b, sign + b);
}

void orc_local_energy_batch(int L, double J1, double J2, int C, int D, const double *theta,
                            int marshall, const int8_t *s, int64_t B, double *eloc,
                            int *n_nbr, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t b = 0; b < B; ++b)
        eloc[b] = orc_local_energy_cnn(L, J1, J2, C, D, theta, marshall, s + b * L * L,
                                       n_nbr ? n_nbr + b : NULL);
}

/* E_loc of one sample with the neighbour evaluations spread over threads;
 * the terms are added in bond order afterwards, so the result does not
 * depend on the thread count. */
double orc_local_energy_cnn_par(int L, double J1, double J2, int C, int D, const double *theta,
                                int marshall, const int8_t *s, int *n_nbr, int nthreads)
{
    const int N = L * L;
    double la; int sa;
    orc_logpsi(L, C, D, theta, marshall, s, &la, &sa);
    double *term = (double *)calloc((size_t)4 * N, sizeof(double));
    double diag = 0.0;
    int nn = 0;
    for (int k = 0; k < 4 * N; ++k) {
        const int i = k / 4, t = k % 4;
        const int j = bond_partner(L, i / L, i % L, t);
        const double J = (t < 2) ? J1 : J2;
        if (s[i] == s[j]) diag += J / 4.0; else { diag -= J / 4.0; ++nn; }
    }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (int k = 0; k < 4 * N; ++k) {
        const int i = k / 4, t = k % 4;
        const int j = bond_partner(L, i / L, i % L, t);
        if (s[i] == s[j]) continue;
        const double J = (t < 2) ? J1 : J2;
        int8_t *sp = (int8_t *)malloc((size_t)N);
        memcpy(sp, s, (size_t)N);
        sp[i] = s[j];
        sp[j] = s[i];
        double lb; int sb;
        orc_logpsi(L, C, D, theta, marshall, sp, &lb, &sb);
        term[k] = (J / 2.0) * ((double)sb / (double)sa) * exp(lb - la);
        free(sp);
    }
    double e = diag;
    for (int k = 0; k < 4 * N; ++k) e += term[k];
    free(term);
    if (n_nbr) *n_nbr = nn;
    return e;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---- log-derivatives O_k = d log|w| / d theta_k (Eq. 5) --------------- */

void orc_log_derivs(int L, int C, int D, const double *theta, const int8_t *s, double *O)
{
    const int N = L * L;
    double *z = (double *)malloc(sizeof(double) * (size_t)(D + 1) * C * N);
    double *g = (double *)malloc(sizeof(double) * (size_t)C * N);   /* d log|w| / d z_l */
    double *gp = (double *)malloc(sizeof(double) * (size_t)C * N);  /* d log|w| / d z_{l-1} */
    double *in = (double *)malloc(sizeof(double) * (size_t)C * N);  /* input of layer l */
    cnn_forward(L, C, D, theta, s, z);
    const double *zD = z + (size_t)D * C * N;
    for (int i = 0; i < C * N; ++i) g[i] = 1.0 / zD[i];
    for (int l = D; l >= 0; --l) {
        const int cin = (l == 0) ? 1 : C;
        const double *W = theta + w_offset(C, l);
        double *dW = O + w_offset(C, l);
        double *db = dW + 9 * C * cin;
        if (l == 0)
            for (int i = 0; i < N; ++i) in[i] = (double)s[i];
        else
            for (int i = 0; i < C * N; ++i) in[i] = silu(z[(size_t)(l - 1) * C * N + i]);
        for (int co = 0; co < C; ++co) {
            double acc = 0.0;
            for (int p = 0; p < N; ++p) acc += g[co * N + p];
            db[co] = acc;
            for (int ci = 0; ci < cin; ++ci)
                for (int ky = 0; ky < 3; ++ky)
                    for (int kx = 0; kx < 3; ++kx) {
                        double a2 = 0.0;
                        for (int y = 0; y < L; ++y)
                            for (int x = 0; x < L; ++x) {
                                int yy = (y + ky - 1 + L) % L, xx = (x + kx - 1 + L) % L;
                                a2 += g[co * N + y * L + x] * in[ci * N + yy * L + xx];
                            }
                        dW[((co * cin + ci) * 3 + ky) * 3 + kx] = a2;
                    }
        }
        if (l == 0) break;
        /* gradient w.r.t. the input activations, then through SiLU */
        for (int i = 0; i < C * N; ++i) gp[i] = 0.0;
        for (int co = 0; co < C; ++co)
            for (int ci = 0; ci < C; ++ci)
                for (int ky = 0; ky < 3; ++ky)
                    for (int kx = 0; kx < 3; ++kx) {
                        const double w = W[((co * C + ci) * 3 + ky) * 3 + kx];
                        for (int y = 0; y < L; ++y)
                            for (int x = 0; x < L; ++x) {
                                int yy = (y + ky - 1 + L) % L, xx = (x + kx - 1 + L) % L;
                                gp[ci * N + yy * L + xx] += w * g[co * N + y * L + x];
                            }
                    }
        const double *zp = z + (size_t)(l - 1) * C * N;
        for (int i = 0; i < C * N; ++i) {
            const double sg = sigmoid(zp[i]);
            g[i] = gp[i] * sg * (1.0 + zp[i] * (1.0 - sg));
        }
    }
    free(z); free(g); free(gp); free(in);
}

void orc_log_derivs_batch(int L, int C, int D, const double *theta, const int8_t *s,
                          int64_t B, double *O, int nthreads)
{
    const int64_t n = orc_num_params(C, D);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t b = 0; b < B; ++b)
        orc_log_derivs(L, C, D, theta, s + b * L * L, O + b * n);
}

/* ---- Stochastic Reconfiguration (Eq. 5-7, Sec. 3.2.2) ----------------- */

/* <O>_k, <E>, G_k = <O_k E> - <E><O_k>, with <.> = (1/m) sum_b. */
void orc_sr_moments(const double *O, const double *E, int64_t m, int64_t n,
                    double *Obar, double *Ebar, double *G)
{
    double eb = 0.0;
    for (int64_t b = 0; b < m; ++b) eb += E[b];
    eb /= (double)m;
    *Ebar = eb;
    for (int64_t k = 0; k < n; ++k) { Obar[k] = 0.0; G[k] = 0.0; }
    for (int64_t b = 0; b < m; ++b)
        for (int64_t k = 0; k < n; ++k) {
            Obar[k] += O[b * n + k];
            G[k] += O[b * n + k] * E[b];
        }
    for (int64_t k = 0; k < n; ++k) {
        Obar[k] /= (double)m;
        G[k] = G[k] / (double)m - eb * Obar[k];
    }
}

/* out = (1/m) O^T (O v) - <O> (<O> . v) + shift v */
void orc_sr_matvec(const double *O, int64_t m, int64_t n, const double *Obar,
                   const double *v, double shift, double *out)
{
    double *t = (double *)malloc(sizeof(double) * (size_t)m);
    for (int64_t b = 0; b < m; ++b) {
        double acc = 0.0;
        for (int64_t k = 0; k < n; ++k) acc += O[b * n + k] * v[k];
        t[b] = acc;
    }
    double c = 0.0;
    for (int64_t k = 0; k < n; ++k) c += Obar[k] * v[k];
    for (int64_t k = 0; k < n; ++k) {
        double acc = 0.0;
        for (int64_t b = 0; b < m; ++b) acc += O[b * n + k] * t[b];
        out[k] = acc / (double)m - Obar[k] * c + shift * v[k];
    }
    free(t);
}

/* The same covariance product with the covariance written in its centred
 * form, M v = (1/m) sum_b (O_b - <O>) ((O_b - <O>) . v): the textbook
 * definition of a sample covariance, equal in real arithmetic to the
 * <O O> - <O><O> of Eq. 7 (Sec. 3.2.2).  In floating point it avoids the
 * cancellation between the two uncentred terms when the column means of O
 * are large against its spread, as they are for log-derivatives of a
 * trained-size network.  The column means are computed here. */
void orc_sr_matvec_centered(const double *O, int64_t m, int64_t n, const double *v, double shift, double *out)
{
    double *c = (double *)calloc((size_t)n, sizeof(double));
    double *d = (double *)malloc(sizeof(double) * (size_t)m);
    for (int64_t b = 0; b < m; ++b)
        for (int64_t k = 0; k < n; ++k) c[k] += O[b * n + k];
    for (int64_t k = 0; k < n; ++k) c[k] /= (double)m;
    for (int64_t b = 0; b < m; ++b) {
        double acc = 0.0;
        for (int64_t k = 0; k < n; ++k) acc += (O[b * n + k] - c[k]) * v[k];
        d[b] = acc;
    }
    for (int64_t k = 0; k < n; ++k) out[k] = 0.0;
    /* out_k accumulates over b in increasing order */
    for (int64_t b = 0; b < m; ++b)
        for (int64_t k = 0; k < n; ++k) out[k] += (O[b * n + k] - c[k]) * d[b];
    for (int64_t k = 0; k < n; ++k) out[k] = out[k] / (double)m + shift * v[k];
    free(c);
    free(d);
}

static double dot(const double *a, const double *b, int64_t n)
{
    double acc = 0.0;
    for (int64_t k = 0; k < n; ++k) acc += a[k] * b[k];
    return acc;
}

/* Plain CG on (M + shift I) x = G from x = 0, exactly `iters` steps (fewer
 * only when the residual or the curvature p.Mp is exactly zero).  Returns ||r|| / ||G|| after the last step. */
double orc_sr_cg(const double *O, int64_t m, int64_t n, const double *Obar, const double *G,
                 double shift, int iters, double *x)
{
    double *r = (double *)malloc(sizeof(double) * (size_t)n);
    double *p = (double *)malloc(sizeof(double) * (size_t)n);
    double *q = (double *)malloc(sizeof(double) * (size_t)n);
    for (int64_t k = 0; k < n; ++k) { x[k] = 0.0; r[k] = G[k]; p[k] = G[k]; }
    const double gg = dot(G, G, n);
    double rr = gg;
    for (int it = 0; it < iters; ++it) {
        if (rr == 0.0) break;           /* already exact: no further step */
        orc_sr_matvec(O, m, n, Obar, p, shift, q);
        const double pq = dot(p, q, n);
        if (pq == 0.0) break;
        const double alpha = rr / pq;
        for (int64_t k = 0; k < n; ++k) { x[k] += alpha * p[k]; r[k] -= alpha * q[k]; }
        const double rr2 = dot(r, r, n);
        const double beta = rr2 / rr;
        for (int64_t k = 0; k < n; ++k) p[k] = r[k] + beta * p[k];
        rr = rr2;
    }
    free(r); free(p); free(q);
    return gg > 0.0 ? sqrt(rr / gg) : 0.0;
}
