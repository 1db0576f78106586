/*
 * Plain CPU FP64 oracle for the DysonNet local estimator.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py may load this library.  It shares no code with the
 * CUDA path: it parses the parameter layout, generates the S4 kernels, runs
 * the network and enumerates the Hamiltonian on its own, in the simplest
 * possible way (direct double sums, no blocking, no fusion).
 *
 * What it computes (paper sections / equations):
 *  - S4 kernel taps: bilinear discretisation (App. "Details on the
 *    implementation of the DysonNet block", Eq. discretization) of a diagonal
 *    state matrix, bidirectional, powers of the discretised eigenvalue taken
 *    with complex pow.  Periodic chains use the circulant image sum in closed
 *    form.
 *  - DysonNet forward (Sec. "DysonNet", Eq. COBALT_recurrence and Eq. wavefunc;
 *    Eq. Dpractical): h^(0)=e*sigma, u=G h, h' = U diag(chi) V u, readout
 *    Omega = A^T P_M G^f sum_l h^(l), log psi = sum_k f(Omega_k).
 *  - Log-amplitude ratio of a flipped configuration by recomputing the whole
 *    network (the quantity ABACUS must reproduce exactly, Theorem 1).
 *  - Local energy (Eq. local-estimator) for the long-range transverse-field
 *    Ising chain (Sec. "Benchmarking") and the J1-J2 Heisenberg chain
 *    (Eq. j1j2_hamiltonian).
 *  - An independent state-space scan (Eq. ssm_discretized read as a diagonal
 *    bidirectional S4) and the Cauchy-kernel resolvent (Eq. resolvent), used
 *    only to pin the taps.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int L, d, s, w, dh, dout, periodic, fkind;
} or_desc;

typedef struct {
    int kind;          /* 0: long-range TFIM, 1: J1-J2 Heisenberg */
    double J, alpha, h; /* TFIM: H = J/Nk sum_{i<j} r^-alpha sz sz + h sum sx */
    double J1, J2;     /* J1-J2: H = J1 sum S_i.S_{i+1} + J2 sum S_i.S_{i+2} */
    int periodic, kac;
} or_ham;

/* ---------------------------------------------------------------- layout -- */

static int s4_size(const or_desc *m) { return 8 * m->d * m->s + m->d; }

static int layer_size(const or_desc *m) {
    int d = m->d, dh = m->dh, W = 2 * m->w + 1;
    return s4_size(m) + W * dh + dh + dh * dh + dh + d * dh + d + 2 * d * d;
}

int or_nparams(const or_desc *m) {
    return m->L * layer_size(m) + s4_size(m) + m->d * m->dout + m->d;
}

typedef struct {
    const double *s4, *kappa, *beta, *W1, *b1, *W2, *b2, *U, *V;
} layer_view;

static layer_view view_layer(const or_desc *m, const double *p, int l /* 1-based */) {
    layer_view v;
    int d = m->d, dh = m->dh, W = 2 * m->w + 1;
    const double *q = p + (size_t)(l - 1) * layer_size(m);
    v.s4 = q; q += s4_size(m);
    v.kappa = q; q += W * dh;
    v.beta = q; q += dh;
    v.W1 = q; q += dh * dh;
    v.b1 = q; q += dh;
    v.W2 = q; q += d * dh;
    v.b2 = q; q += d;
    v.U = q; q += d * d;
    v.V = q;
    return v;
}

static const double *final_s4(const or_desc *m, const double *p) {
    return p + (size_t)m->L * layer_size(m);
}
static const double *final_A(const or_desc *m, const double *p) {
    return final_s4(m, p) + s4_size(m);
}
static const double *final_e(const or_desc *m, const double *p) {
    return final_A(m, p) + m->d * m->dout;
}

/* ------------------------------------------------------------- S4 kernel -- */

/* Discretised eigenvalue and input of mode n of channel c (Eq. discretization,
 * diagonal case): lam_bar = (1 + dt/2 Lam)/(1 - dt/2 Lam), B_bar = dt B/(1 - dt/2 Lam). */
static void s4_mode(const or_desc *m, const double *blk, int c, int n,
                    double complex *lam_bar, double complex *b_bar,
                    double complex *cf, double complex *cb) {
    int d = m->d, s = m->s;
    const double *lre = blk, *lim = lre + d * s, *logdt = lim + d * s;
    const double *bre = logdt + d, *bim = bre + d * s;
    const double *cfre = bim + d * s, *cfim = cfre + d * s;
    const double *cbre = cfim + d * s, *cbim = cbre + d * s;
    int k = c * s + n;
    double dt = exp(logdt[c]);
    double complex lam = lre[k] + I * lim[k];
    double complex den = 1.0 - 0.5 * dt * lam;
    *lam_bar = (1.0 + 0.5 * dt * lam) / den;
    *b_bar = dt * (bre[k] + I * bim[k]) / den;
    *cf = cfre[k] + I * cfim[k];
    *cb = cbre[k] + I * cbim[k];
}

/* Open chain: taps g[(r + N - 1) * d + c] for r in (-N, N).
 *   r >= 0: Re sum_n Cf B_bar lam_bar^r ;  r < 0: Re sum_n Cb B_bar lam_bar^|r|.
 * Periodic chain: circulant taps g[r * d + c], r in [0, N): the open kernel summed
 * over all periodic images, in closed form
 *   Re sum_n B_bar [Cf lam^r + Cb lam^(N-r)] / (1 - lam^N). */
void or_s4_taps(const or_desc *m, const double *blk, int N, int periodic, double *g) {
    int d = m->d, s = m->s;
    int R = periodic ? N : 2 * N - 1;
    memset(g, 0, sizeof(double) * (size_t)R * d);
    for (int c = 0; c < d; ++c) {
        for (int n = 0; n < s; ++n) {
            double complex lb, bb, cf, cb;
            s4_mode(m, blk, c, n, &lb, &bb, &cf, &cb);
            if (!periodic) {
                for (int r = -(N - 1); r <= N - 1; ++r) {
                    double complex t;
                    if (r >= 0) t = cf * bb * cpow(lb, (double)r);
                    else t = cb * bb * cpow(lb, (double)(-r));
                    g[(size_t)(r + N - 1) * d + c] += creal(t);
                }
            } else {
                double complex lN = cpow(lb, (double)N);
                for (int r = 0; r < N; ++r) {
                    double complex t = bb * (cf * cpow(lb, (double)r) + cb * cpow(lb, (double)(N - r))) / (1.0 - lN);
                    g[(size_t)r * d + c] += creal(t);
                }
            }
        }
    }
}

/* Resolvent (Eq. resolvent, diagonal A): Gc(z_k) = sum_n Cf_n B_bar_n / (1 - z_k lam_n),
 * z_k = exp(2 pi i k / N), forward direction only.  out[(k*d + c)*2 + {0,1}] = re, im. */
void or_s4_resolvent(const or_desc *m, const double *blk, int N, double *out) {
    int d = m->d, s = m->s;
    for (int k = 0; k < N; ++k) {
        double complex z = cexp(I * 2.0 * M_PI * k / N);
        for (int c = 0; c < d; ++c) {
            double complex acc = 0;
            for (int n = 0; n < s; ++n) {
                double complex lb, bb, cf, cb;
                s4_mode(m, blk, c, n, &lb, &bb, &cf, &cb);
                acc += cf * bb / (1.0 - z * lb);
            }
            out[((size_t)k * d + c) * 2 + 0] = creal(acc);
            out[((size_t)k * d + c) * 2 + 1] = cimag(acc);
        }
    }
}

/* Complex (pre-Re) forward circulant kernel, for the resolvent pin:
 * out[(r*d + c)*2 + {0,1}] = sum_n Cf B_bar lam^r / (1 - lam^N). */
void or_s4_circulant_fwd_complex(const or_desc *m, const double *blk, int N, double *out) {
    int d = m->d, s = m->s;
    for (int r = 0; r < N; ++r)
        for (int c = 0; c < d; ++c) {
            double complex acc = 0;
            for (int n = 0; n < s; ++n) {
                double complex lb, bb, cf, cb;
                s4_mode(m, blk, c, n, &lb, &bb, &cf, &cb);
                acc += cf * bb * cpow(lb, (double)r) / (1.0 - cpow(lb, (double)N));
            }
            out[((size_t)r * d + c) * 2 + 0] = creal(acc);
            out[((size_t)r * d + c) * 2 + 1] = cimag(acc);
        }
}

/* Independent state-space scan of an open chain (no powers):
 *   x_i = lam x_{i-1} + B_bar h_i,          y_fwd_i = Re sum_n Cf_n x_i,n
 *   z_i = lam (z_{i+1} + B_bar h_{i+1}),     y_bwd_i = Re sum_n Cb_n z_i,n
 * u = y_fwd + y_bwd.  h, u: [N][d]. */
void or_s4_scan(const or_desc *m, const double *blk, int N, const double *h, double *u) {
    int d = m->d, s = m->s;
    memset(u, 0, sizeof(double) * (size_t)N * d);
    for (int c = 0; c < d; ++c)
        for (int n = 0; n < s; ++n) {
            double complex lb, bb, cf, cb;
            s4_mode(m, blk, c, n, &lb, &bb, &cf, &cb);
            double complex x = 0;
            for (int i = 0; i < N; ++i) {
                x = lb * x + bb * h[(size_t)i * d + c];
                u[(size_t)i * d + c] += creal(cf * x);
            }
            double complex z = 0;
            for (int i = N - 1; i >= 0; --i) {
                if (i + 1 < N) z = lb * (z + bb * h[(size_t)(i + 1) * d + c]);
                u[(size_t)i * d + c] += creal(cb * z);
            }
        }
}

/* ----------------------------------------------------------- the network -- */

typedef struct {
    int N;
    double *taps;   /* L layer kernels, each R*d */
    double *omega;  /* [N][d] pooling weights (1/N) sum_k g^f_{k-i} */
    int R;
} or_plan;

static void plan_make(const or_desc *m, const double *p, int N, or_plan *pl) {
    int d = m->d;
    pl->N = N;
    pl->R = m->periodic ? N : 2 * N - 1;
    pl->taps = (double *)malloc(sizeof(double) * (size_t)m->L * pl->R * d);
    for (int l = 1; l <= m->L; ++l) {
        layer_view v = view_layer(m, p, l);
        or_s4_taps(m, v.s4, N, m->periodic, pl->taps + (size_t)(l - 1) * pl->R * d);
    }
    double *gf = (double *)malloc(sizeof(double) * (size_t)pl->R * d);
    or_s4_taps(m, final_s4(m, p), N, m->periodic, gf);
    pl->omega = (double *)malloc(sizeof(double) * (size_t)N * d);
    /* (P_M G^f h)_c = (1/N) sum_k sum_i g^f_{k-i,c} h_{i,c} = sum_i omega_{i,c} h_{i,c} */
    for (int i = 0; i < N; ++i)
        for (int c = 0; c < d; ++c) {
            double acc = 0;
            for (int k = 0; k < N; ++k) {
                if (m->periodic) acc += gf[(size_t)(((k - i) % N + N) % N) * d + c];
                else acc += gf[(size_t)(k - i + N - 1) * d + c];
            }
            pl->omega[(size_t)i * d + c] = acc / N;
        }
    free(gf);
}

static void plan_free(or_plan *pl) {
    free(pl->taps);
    free(pl->omega);
}

static double gelu(double x) { return 0.5 * x * (1.0 + erf(x / sqrt(2.0))); }

static double log_cosh(double x) {
    double a = fabs(x);
    return a + log1p(exp(-2.0 * a)) - log(2.0);
}

/* Neumaier compensated accumulation. */
typedef struct { double sum, comp; } nsum;
static void nsum_add(nsum *a, double x) {
    double t = a->sum + x;
    if (fabs(a->sum) >= fabs(x)) a->comp += (a->sum - t) + x;
    else a->comp += (x - t) + a->sum;
    a->sum = t;
}

/* Spin at site i, zero off an open chain, wrapped on a ring. */
static double spin_at(const or_desc *m, const int8_t *sp, int N, int i) {
    if (m->periodic) return (double)sp[((i % N) + N) % N];
    if (i < 0 || i >= N) return 0.0;
    return (double)sp[i];
}

/* chi^(l)_i = W2 GELU(W1 phi_i + b1) + b2,  phi_i = sum_{r=-w..w} kappa_r sigma_{i+r} + beta. */
static void local_chi(const or_desc *m, const layer_view *v, const int8_t *sp, int N, int i,
                      double *chi, double *work) {
    int d = m->d, dh = m->dh, w = m->w;
    double *phi = work, *a = work + dh;
    for (int e = 0; e < dh; ++e) {
        double acc = v->beta[e];
        for (int r = -w; r <= w; ++r) acc += v->kappa[(r + w) * dh + e] * spin_at(m, sp, N, i + r);
        phi[e] = acc;
    }
    for (int e = 0; e < dh; ++e) {
        double acc = v->b1[e];
        for (int f = 0; f < dh; ++f) acc += v->W1[e * dh + f] * phi[f];
        a[e] = gelu(acc);
    }
    for (int c = 0; c < d; ++c) {
        double acc = v->b2[c];
        for (int e = 0; e < dh; ++e) acc += v->W2[c * dh + e] * a[e];
        chi[c] = acc;
    }
}

/* Whole-network forward for one configuration.  Returns log psi; writes Omega[dout]. */
static double forward_one(const or_desc *m, const double *p, const or_plan *pl,
                          const int8_t *sp, double *Omega) {
    int N = pl->N, d = m->d, dh = m->dh;
    double *h = (double *)malloc(sizeof(double) * (size_t)N * d);
    double *u = (double *)malloc(sizeof(double) * (size_t)N * d);
    double *chi = (double *)malloc(sizeof(double) * d);
    double *y = (double *)malloc(sizeof(double) * d);
    double *t = (double *)malloc(sizeof(double) * d);
    double *work = (double *)malloc(sizeof(double) * 2 * dh);
    nsum *pool = (nsum *)calloc(d, sizeof(nsum));
    const double *e = final_e(m, p), *A = final_A(m, p);

    for (int i = 0; i < N; ++i)
        for (int c = 0; c < d; ++c) h[(size_t)i * d + c] = e[c] * (double)sp[i];
    for (int i = 0; i < N; ++i)
        for (int c = 0; c < d; ++c) nsum_add(&pool[c], pl->omega[(size_t)i * d + c] * h[(size_t)i * d + c]);

    for (int l = 1; l <= m->L; ++l) {
        layer_view v = view_layer(m, p, l);
        const double *g = pl->taps + (size_t)(l - 1) * pl->R * d;
        /* u = G h (channel-wise Toeplitz / circulant convolution) */
        for (int i = 0; i < N; ++i)
            for (int c = 0; c < d; ++c) {
                double acc = 0;
                for (int j = 0; j < N; ++j) {
                    double gr = m->periodic ? g[(size_t)(((i - j) % N + N) % N) * d + c]
                                            : g[(size_t)(i - j + N - 1) * d + c];
                    acc += gr * h[(size_t)j * d + c];
                }
                u[(size_t)i * d + c] = acc;
            }
        /* h_i = U diag(chi_i) V u_i */
        for (int i = 0; i < N; ++i) {
            local_chi(m, &v, sp, N, i, chi, work);
            for (int a = 0; a < d; ++a) {
                double acc = 0;
                for (int b = 0; b < d; ++b) acc += v.V[a * d + b] * u[(size_t)i * d + b];
                y[a] = acc;
                t[a] = chi[a] * y[a];
            }
            for (int a = 0; a < d; ++a) {
                double acc = 0;
                for (int b = 0; b < d; ++b) acc += v.U[a * d + b] * t[b];
                h[(size_t)i * d + a] = acc;
            }
        }
        for (int i = 0; i < N; ++i)
            for (int c = 0; c < d; ++c) nsum_add(&pool[c], pl->omega[(size_t)i * d + c] * h[(size_t)i * d + c]);
    }
    double logpsi = 0;
    for (int k = 0; k < m->dout; ++k) {
        double acc = 0;
        for (int c = 0; c < d; ++c) acc += A[c * m->dout + k] * (pool[c].sum + pool[c].comp);
        Omega[k] = acc;
        logpsi += (m->fkind == 0) ? log_cosh(acc) : acc;
    }
    free(h); free(u); free(chi); free(y); free(t); free(work); free(pool);
    return logpsi;
}

/* log psi and Omega for B configurations (OpenMP over samples). */
void or_logpsi(const or_desc *m, const double *p, int N, const int8_t *spins, int B,
               double *logpsi, double *Omega) {
    or_plan pl;
    plan_make(m, p, N, &pl);
#pragma omp parallel for schedule(dynamic)
    for (int b = 0; b < B; ++b) {
        double om[64];
        double lp = forward_one(m, p, &pl, spins + (size_t)b * N, om);
        if (logpsi) logpsi[b] = lp;
        if (Omega)
            for (int k = 0; k < m->dout; ++k) Omega[(size_t)b * m->dout + k] = om[k];
    }
    plan_free(&pl);
}

/* Taps of every layer kernel (L blocks of R*d) and the pooling weights omega [N][d]. */
void or_plan_export(const or_desc *m, const double *p, int N, double *taps, double *omega) {
    or_plan pl;
    plan_make(m, p, N, &pl);
    if (taps) memcpy(taps, pl.taps, sizeof(double) * (size_t)m->L * pl.R * m->d);
    if (omega) memcpy(omega, pl.omega, sizeof(double) * (size_t)N * m->d);
    plan_free(&pl);
}

/* log psi(sigma') - log psi(sigma) by two full forward passes per flip set.
 * sites[f*2 + {0,1}]: flipped sites, -1 = unused. */
void or_dlogpsi(const or_desc *m, const double *p, int N, const int8_t *spins, int B,
                const int32_t *sample, const int32_t *sites, int F, double *out) {
    or_plan pl;
    plan_make(m, p, N, &pl);
    double *base = (double *)malloc(sizeof(double) * (size_t)B);
    char *need = (char *)calloc((size_t)B, 1);
    for (int f = 0; f < F; ++f) need[sample[f]] = 1;
#pragma omp parallel for schedule(dynamic)
    for (int b = 0; b < B; ++b) {
        double om[64];
        if (need[b]) base[b] = forward_one(m, p, &pl, spins + (size_t)b * N, om);
    }
#pragma omp parallel for schedule(dynamic)
    for (int f = 0; f < F; ++f) {
        int8_t *sp = (int8_t *)malloc((size_t)N);
        double om[64];
        memcpy(sp, spins + (size_t)sample[f] * N, (size_t)N);
        for (int q = 0; q < 2; ++q) {
            int j = sites[f * 2 + q];
            if (j >= 0) sp[j] = (int8_t)(-sp[j]);
        }
        out[f] = forward_one(m, p, &pl, sp, om) - base[sample[f]];
        free(sp);
    }
    free(base);
    free(need);
    plan_free(&pl);
}

/* ------------------------------------------------ parameter derivatives -- */
/* Per-configuration derivative of log psi with respect to every parameter (the
 * log-derivatives O_k of the variational parameters used by the energy gradient and
 * stochastic reconfiguration, Sec. "Variational Monte Carlo").  Plain reverse-mode
 * differentiation of forward_one written out by hand, in the forward's order
 * reversed; the result uses the parameter layout of the weights vector. */

static double gelu_prime(double x) {
    return 0.5 * (1.0 + erf(x / sqrt(2.0))) + x * exp(-0.5 * x * x) / sqrt(2.0 * M_PI);
}

/* d J / d(S4 block) for J = sum_r dg[r][c] g[r][c] (taps layout of or_s4_taps).
 * J is the real part of an analytic function F of each complex parameter z, so
 * dJ/dRe z = Re F'(z) and dJ/dIm z = -Im F'(z). */
static void s4_block_grad(const or_desc *m, const double *blk, int N, int periodic, const double *dg, double *gblk) {
    int d = m->d, s = m->s;
    double *glre = gblk, *glim = glre + d * s, *glogdt = glim + d * s;
    double *gbre = glogdt + d, *gbim = gbre + d * s;
    double *gcfre = gbim + d * s, *gcfim = gcfre + d * s;
    double *gcbre = gcfim + d * s, *gcbim = gcbre + d * s;
    const double *lre = blk, *lim = lre + d * s, *logdt = lim + d * s;
    const double *bre = logdt + d, *bim = bre + d * s;
    for (int c = 0; c < d; ++c) {
        double dt = exp(logdt[c]);
        double gdt = 0.0;
        for (int n = 0; n < s; ++n) {
            int k = c * s + n;
            double complex lb, bb, cf, cb;
            s4_mode(m, blk, c, n, &lb, &bb, &cf, &cb);
            double complex lam = lre[k] + I * lim[k], Bc = bre[k] + I * bim[k];
            double complex den = 1.0 - 0.5 * dt * lam;
            double complex wf, wb, Q, E;   /* dF/dCf, dF/dCb, dF/dB_bar, dF/dlam_bar */
            if (!periodic) {
                double complex Gp = 0, Gm = 0, Hp = 0, Hm = 0;
                for (int r = -(N - 1); r <= N - 1; ++r) {
                    double x = dg[(size_t)(r + N - 1) * d + c];
                    int q = r < 0 ? -r : r;
                    double complex pw = cpow(lb, (double)q);
                    double complex pw1 = q > 0 ? (double)q * cpow(lb, (double)(q - 1)) : 0.0;
                    if (r >= 0) { Gp += x * pw; Hp += x * pw1; }
                    else { Gm += x * pw; Hm += x * pw1; }
                }
                wf = bb * Gp;
                wb = bb * Gm;
                Q = cf * Gp + cb * Gm;
                E = bb * (cf * Hp + cb * Hm);
            } else {
                double complex lN = cpow(lb, (double)N), inv = 1.0 / (1.0 - lN);
                double complex Sf = 0, Sb = 0, Sf1 = 0, Sb1 = 0;
                for (int r = 0; r < N; ++r) {
                    double x = dg[(size_t)r * d + c];
                    Sf += x * cpow(lb, (double)r);
                    Sb += x * cpow(lb, (double)(N - r));
                    if (r > 0) Sf1 += x * (double)r * cpow(lb, (double)(r - 1));
                    Sb1 += x * (double)(N - r) * cpow(lb, (double)(N - r - 1));
                }
                double complex S = cf * Sf + cb * Sb, S1 = cf * Sf1 + cb * Sb1;
                wf = bb * Sf * inv;
                wb = bb * Sb * inv;
                Q = S * inv;
                E = bb * (S1 * inv + S * (double)N * cpow(lb, (double)(N - 1)) * inv * inv);
            }
            /* lam_bar = (1 + dt lam/2)/den, B_bar = dt B/den, den = 1 - dt lam/2 */
            double complex den2 = den * den;
            double complex dLam = E * dt / den2 + Q * dt * dt * Bc / (2.0 * den2);
            double complex dB = Q * dt / den;
            double complex dDt = E * lam / den2 + Q * Bc / den2;
            glre[k] = creal(dLam);
            glim[k] = -cimag(dLam);
            gbre[k] = creal(dB);
            gbim[k] = -cimag(dB);
            gcfre[k] = creal(wf);
            gcfim[k] = -cimag(wf);
            gcbre[k] = creal(wb);
            gcbim[k] = -cimag(wb);
            gdt += creal(dDt);
        }
        glogdt[c] = gdt * dt;
    }
}

typedef struct {
    double *s4, *kappa, *beta, *W1, *b1, *W2, *b2, *U, *V;
} layer_grad_view;

static layer_grad_view view_layer_grad(const or_desc *m, double *p, int l) {
    layer_view v = view_layer(m, p, l);
    layer_grad_view g = {(double *)v.s4, (double *)v.kappa, (double *)v.beta, (double *)v.W1, (double *)v.b1,
                         (double *)v.W2, (double *)v.b2, (double *)v.U, (double *)v.V};
    return g;
}

/* log psi of one configuration and its derivative with respect to all parameters. */
static double grad_one(const or_desc *m, const double *p, const or_plan *pl, const int8_t *sp, double *grad) {
    int N = pl->N, d = m->d, dh = m->dh, L = m->L, w = m->w, R = pl->R;
    size_t Nd = (size_t)N * d, Ndh = (size_t)N * dh;
    double *h = (double *)calloc((size_t)(L + 1) * Nd, sizeof(double));   /* h^(0..L) */
    double *u = (double *)calloc((size_t)L * Nd, sizeof(double));         /* u^(1..L) */
    double *y = (double *)calloc((size_t)L * Nd, sizeof(double));
    double *chi = (double *)calloc((size_t)L * Nd, sizeof(double));
    double *phi = (double *)calloc((size_t)L * Ndh, sizeof(double));
    double *z = (double *)calloc((size_t)L * Ndh, sizeof(double));        /* W1 phi + b1 */
    double *dh_ = (double *)calloc(Nd, sizeof(double)), *du = (double *)calloc(Nd, sizeof(double));
    double *dg = (double *)calloc((size_t)R * d, sizeof(double));
    double *domega = (double *)calloc(Nd, sizeof(double));
    double *tmp = (double *)calloc((size_t)3 * (d > dh ? d : dh), sizeof(double));
    double *pool = (double *)malloc(sizeof(double) * (size_t)d), *acol = (double *)malloc(sizeof(double) * (size_t)d);
    double fp[64];
    const double *e = final_e(m, p), *A = final_A(m, p);
    memset(grad, 0, sizeof(double) * (size_t)or_nparams(m));

    /* forward, keeping every intermediate */
    for (int i = 0; i < N; ++i)
        for (int c = 0; c < d; ++c) h[(size_t)i * d + c] = e[c] * (double)sp[i];
    for (int l = 1; l <= L; ++l) {
        layer_view v = view_layer(m, p, l);
        const double *g = pl->taps + (size_t)(l - 1) * R * d;
        const double *hp = h + (size_t)(l - 1) * Nd;
        double *ul = u + (size_t)(l - 1) * Nd, *yl = y + (size_t)(l - 1) * Nd, *cl = chi + (size_t)(l - 1) * Nd;
        double *hl = h + (size_t)l * Nd, *pf = phi + (size_t)(l - 1) * Ndh, *zl = z + (size_t)(l - 1) * Ndh;
        for (int i = 0; i < N; ++i)
            for (int c = 0; c < d; ++c) {
                double acc = 0;
                for (int j = 0; j < N; ++j) {
                    double gr = m->periodic ? g[(size_t)(((i - j) % N + N) % N) * d + c] : g[(size_t)(i - j + N - 1) * d + c];
                    acc += gr * hp[(size_t)j * d + c];
                }
                ul[(size_t)i * d + c] = acc;
            }
        for (int i = 0; i < N; ++i) {
            double *ph = pf + (size_t)i * dh, *zz = zl + (size_t)i * dh, *ch = cl + (size_t)i * d;
            for (int f = 0; f < dh; ++f) {
                double acc = v.beta[f];
                for (int r = -w; r <= w; ++r) acc += v.kappa[(r + w) * dh + f] * spin_at(m, sp, N, i + r);
                ph[f] = acc;
            }
            for (int f = 0; f < dh; ++f) {
                double acc = v.b1[f];
                for (int q = 0; q < dh; ++q) acc += v.W1[f * dh + q] * ph[q];
                zz[f] = acc;
            }
            for (int c = 0; c < d; ++c) {
                double acc = v.b2[c];
                for (int f = 0; f < dh; ++f) acc += v.W2[c * dh + f] * gelu(zz[f]);
                ch[c] = acc;
            }
            for (int a = 0; a < d; ++a) {
                double acc = 0;
                for (int b = 0; b < d; ++b) acc += v.V[a * d + b] * ul[(size_t)i * d + b];
                yl[(size_t)i * d + a] = acc;
            }
            for (int a = 0; a < d; ++a) {
                double acc = 0;
                for (int b = 0; b < d; ++b) acc += v.U[a * d + b] * ch[b] * yl[(size_t)i * d + b];
                hl[(size_t)i * d + a] = acc;
            }
        }
    }
    for (int c = 0; c < d; ++c) {
        nsum acc = {0, 0};
        for (int l = 0; l <= L; ++l)
            for (int i = 0; i < N; ++i) nsum_add(&acc, pl->omega[(size_t)i * d + c] * h[(size_t)l * Nd + (size_t)i * d + c]);
        pool[c] = acc.sum + acc.comp;
    }
    double logpsi = 0;
    for (int k = 0; k < m->dout; ++k) {
        double acc = 0;
        for (int c = 0; c < d; ++c) acc += A[c * m->dout + k] * pool[c];
        logpsi += (m->fkind == 0) ? log_cosh(acc) : acc;
        fp[k] = (m->fkind == 0) ? tanh(acc) : 1.0;
    }

    /* readout: dA, the coefficient a_c of the pooled sum, d omega */
    double *gA = grad + (final_A(m, p) - p);
    for (int c = 0; c < d; ++c) {
        double acc = 0;
        for (int k = 0; k < m->dout; ++k) {
            gA[c * m->dout + k] = pool[c] * fp[k];
            acc += A[c * m->dout + k] * fp[k];
        }
        acol[c] = acc;
    }
    for (int i = 0; i < N; ++i)
        for (int c = 0; c < d; ++c) {
            double acc = 0;
            for (int l = 0; l <= L; ++l) acc += h[(size_t)l * Nd + (size_t)i * d + c];
            domega[(size_t)i * d + c] = acol[c] * acc;
        }
    /* layers in reverse */
    for (int i = 0; i < N; ++i)
        for (int c = 0; c < d; ++c) dh_[(size_t)i * d + c] = pl->omega[(size_t)i * d + c] * acol[c];
    for (int l = L; l >= 1; --l) {
        layer_view v = view_layer(m, p, l);
        layer_grad_view gv = view_layer_grad(m, grad, l);
        const double *g = pl->taps + (size_t)(l - 1) * R * d;
        const double *hp = h + (size_t)(l - 1) * Nd;
        const double *ul = u + (size_t)(l - 1) * Nd, *yl = y + (size_t)(l - 1) * Nd, *cl = chi + (size_t)(l - 1) * Nd;
        const double *pf = phi + (size_t)(l - 1) * Ndh, *zl = z + (size_t)(l - 1) * Ndh;
        double *dt_ = tmp, *dchi = tmp + d, *dy = tmp + 2 * d;
        for (int i = 0; i < N; ++i) {
            const double *dhi = dh_ + (size_t)i * d, *ch = cl + (size_t)i * d, *yi = yl + (size_t)i * d;
            /* h_i = U (chi_i . y_i) */
            for (int b = 0; b < d; ++b) {
                double acc = 0;
                for (int a = 0; a < d; ++a) {
                    acc += v.U[a * d + b] * dhi[a];
                    gv.U[a * d + b] += dhi[a] * ch[b] * yi[b];
                }
                dt_[b] = acc;
            }
            for (int b = 0; b < d; ++b) {
                dchi[b] = dt_[b] * yi[b];
                dy[b] = dt_[b] * ch[b];
            }
            /* y_i = V u_i */
            for (int b = 0; b < d; ++b) {
                double acc = 0;
                for (int a = 0; a < d; ++a) {
                    acc += v.V[a * d + b] * dy[a];
                    gv.V[a * d + b] += dy[a] * ul[(size_t)i * d + b];
                }
                du[(size_t)i * d + b] = acc;
            }
            /* chi_i = W2 gelu(z_i) + b2, z_i = W1 phi_i + b1, phi_i = sum_r kappa_r sigma_{i+r} + beta */
            const double *zz = zl + (size_t)i * dh, *ph = pf + (size_t)i * dh;
            double *dz = (double *)malloc(sizeof(double) * (size_t)dh), *dphi = (double *)malloc(sizeof(double) * (size_t)dh);
            for (int c = 0; c < d; ++c) gv.b2[c] += dchi[c];
            for (int f = 0; f < dh; ++f) {
                double acc = 0, gz = gelu(zz[f]);
                for (int c = 0; c < d; ++c) {
                    gv.W2[c * dh + f] += dchi[c] * gz;
                    acc += v.W2[c * dh + f] * dchi[c];
                }
                dz[f] = acc * gelu_prime(zz[f]);
            }
            for (int f = 0; f < dh; ++f) {
                gv.b1[f] += dz[f];
                for (int q = 0; q < dh; ++q) gv.W1[f * dh + q] += dz[f] * ph[q];
            }
            for (int q = 0; q < dh; ++q) {
                double acc = 0;
                for (int f = 0; f < dh; ++f) acc += v.W1[f * dh + q] * dz[f];
                dphi[q] = acc;
            }
            for (int q = 0; q < dh; ++q) {
                gv.beta[q] += dphi[q];
                for (int r = -w; r <= w; ++r) gv.kappa[(r + w) * dh + q] += dphi[q] * spin_at(m, sp, N, i + r);
            }
            free(dz);
            free(dphi);
        }
        /* u = G h^(l-1): taps and the field below */
        memset(dg, 0, sizeof(double) * (size_t)R * d);
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j)
                for (int c = 0; c < d; ++c) {
                    size_t row = m->periodic ? (size_t)(((i - j) % N + N) % N) : (size_t)(i - j + N - 1);
                    dg[row * d + c] += du[(size_t)i * d + c] * hp[(size_t)j * d + c];
                }
        s4_block_grad(m, v.s4, N, m->periodic, dg, gv.s4);
        for (int j = 0; j < N; ++j)
            for (int c = 0; c < d; ++c) {
                double acc = pl->omega[(size_t)j * d + c] * acol[c];
                for (int i = 0; i < N; ++i) {
                    double gr = m->periodic ? g[(size_t)(((i - j) % N + N) % N) * d + c] : g[(size_t)(i - j + N - 1) * d + c];
                    acc += gr * du[(size_t)i * d + c];
                }
                dh_[(size_t)j * d + c] = acc;
            }
    }
    /* h^(0) = e sigma */
    double *ge = grad + (final_e(m, p) - p);
    for (int c = 0; c < d; ++c) {
        double acc = 0;
        for (int i = 0; i < N; ++i) acc += dh_[(size_t)i * d + c] * (double)sp[i];
        ge[c] = acc;
    }
    /* omega_{i,c} = (1/N) sum_k g^f_{k-i,c} */
    memset(dg, 0, sizeof(double) * (size_t)R * d);
    for (int i = 0; i < N; ++i)
        for (int k = 0; k < N; ++k)
            for (int c = 0; c < d; ++c) {
                size_t row = m->periodic ? (size_t)(((k - i) % N + N) % N) : (size_t)(k - i + N - 1);
                dg[row * d + c] += domega[(size_t)i * d + c] / N;
            }
    s4_block_grad(m, final_s4(m, p), N, m->periodic, dg, grad + (final_s4(m, p) - p));
    free(h); free(u); free(y); free(chi); free(phi); free(z); free(dh_); free(du); free(dg); free(domega); free(tmp);
    free(pool); free(acol);
    return logpsi;
}

/* log psi [B] and d log psi / d theta [B][nparams] (OpenMP over samples). */
void or_grad_logpsi(const or_desc *m, const double *p, int N, const int8_t *spins, int B, double *logpsi,
                    double *grad) {
    or_plan pl;
    plan_make(m, p, N, &pl);
    size_t np = (size_t)or_nparams(m);
#pragma omp parallel for schedule(dynamic)
    for (int b = 0; b < B; ++b) {
        double lp = grad_one(m, p, &pl, spins + (size_t)b * N, grad + (size_t)b * np);
        if (logpsi) logpsi[b] = lp;
    }
    plan_free(&pl);
}

/* ---------------------------------------------------------- Hamiltonians -- */

static double tfim_coupling(const or_ham *H, int N, int i, int j) {
    int r = abs(i - j);
    if (H->periodic && N - r < r) r = N - r;
    double norm = 1.0;
    if (H->kac) {
        norm = 0.0;
        for (int q = 1; q <= N / 2; ++q) norm += 2.0 * pow((double)q, -H->alpha);
    }
    return H->J * pow((double)r, -H->alpha) / norm;
}

/* Diagonal matrix element <sigma|H|sigma>. */
double or_diag(const or_ham *H, int N, const int8_t *sp) {
    double acc = 0;
    if (H->kind == 0) {
        for (int i = 0; i < N; ++i)
            for (int j = i + 1; j < N; ++j) acc += tfim_coupling(H, N, i, j) * sp[i] * sp[j];
    } else {
        for (int b = 1; b <= 2; ++b) {
            double Jb = (b == 1) ? H->J1 : H->J2;
            int imax = H->periodic ? N : N - b;
            for (int i = 0; i < imax; ++i) acc += Jb * 0.25 * sp[i] * sp[(i + b) % N];
        }
    }
    return acc;
}

/* Local energy E_loc(sigma) = sum_sigma' <sigma|H|sigma'> psi(sigma')/psi(sigma),
 * each ratio by full recompute.  Off-diagonal elements:
 *   TFIM: h for every single flip;  J1-J2: J_b/2 for every antialigned pair (i, i+b). */
void or_eloc(const or_desc *m, const double *p, const or_ham *H, int N, const int8_t *spins,
             int B, double *eloc) {
    or_plan pl;
    plan_make(m, p, N, &pl);
#pragma omp parallel for schedule(dynamic)
    for (int b = 0; b < B; ++b) {
        const int8_t *sp = spins + (size_t)b * N;
        int8_t *q = (int8_t *)malloc((size_t)N);
        double om[64];
        double lp0 = forward_one(m, p, &pl, sp, om);
        double e = or_diag(H, N, sp);
        if (H->kind == 0) {
            for (int i = 0; i < N; ++i) {
                memcpy(q, sp, (size_t)N);
                q[i] = (int8_t)(-q[i]);
                e += H->h * exp(forward_one(m, p, &pl, q, om) - lp0);
            }
        } else {
            for (int bb = 1; bb <= 2; ++bb) {
                double Jb = (bb == 1) ? H->J1 : H->J2;
                int imax = H->periodic ? N : N - bb;
                for (int i = 0; i < imax; ++i) {
                    int j = (i + bb) % N;
                    if (sp[i] == sp[j]) continue;
                    memcpy(q, sp, (size_t)N);
                    q[i] = (int8_t)(-q[i]);
                    q[j] = (int8_t)(-q[j]);
                    e += Jb * 0.5 * exp(forward_one(m, p, &pl, q, om) - lp0);
                }
            }
        }
        eloc[b] = e;
        free(q);
    }
    plan_free(&pl);
}
