/*
 * FP64 CPU oracle for decentralized coordinate-descent (CD) data detection and precoding
 * (K. Li, O. Castaneda, C. Jeon, J. R. Cavallaro, C. Studer, "Decentralized Coordinate-Descent Data
 * Detection and Precoding for Massive MU-MIMO", arXiv 1902.08653).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's CPU-baseline
 * leg load this file.  The CUDA library shares no code, header, table or helper with it.
 *
 * Plain, slow, obviously correct: one subcarrier, one cluster, one symbol at a time, in the order
 * and notation of the paper's algorithms, in double precision (C99 double _Complex).  Each function
 * cites the passage it follows.
 *
 * Array layouts (row-major; complex = interleaved re/im, i.e. double _Complex):
 *   H    [n_sc][U][B]      row u is column h_u of the B x U uplink matrix H^ul; for cluster c with
 *                          antenna offset o_c, h_{u,c} = H[f][u][o_c .. o_c+B_c-1].
 *   Y    [n_sc][n_sym][B]  uplink receive vectors y (H fixed over the n_sym symbols).
 *   S    [n_sc][n_sym][U]  downlink symbol vectors s.
 *   N0   [n_sc]            noise variance per receive antenna.
 *   Xhat [n_sc][n_sym][U]  fused uplink estimate; Xc [n_sc][C][n_sym][U] per-cluster estimates.
 *   Xdl  [n_sc][n_sym][B]  stacked downlink beamforming vector [x_1; ...; x_C].
 * Clusters are contiguous antenna ranges in order: o_0 = 0, o_{c+1} = o_c + B_c (Sec. II-A).
 *
 * Readings where the paper is silent (each repeated where it is used):
 *   - fusion weights (Sec. III): lambda_c = sigma_c^{-2} / sum_c' sigma_c'^{-2}, with the
 *     post-equalization noise variance taken as sigma_c^2 = (N0/U) sum_u (||h_{u,c}||^2 + N0/Ex)^{-1};
 *     the common factor N0/U cancels, so lambda is evaluated without it (also valid at N0 = 0).
 *   - a zero column with N0 = 0: m_{u,c} := 0 (Alg. 1) and p_{u,c} := 0 (Alg. 2), i.e. that user is
 *     skipped; a zero local beamformer is left at zero by the normalization.
 *   - per-cluster power: rho_c = rho / sqrt(C) (Sec. IV-B, rho_c^2 = rho^2 / C), also for uneven B_c.
 *   - the garbled transposes of Alg. 2 are read as Eq. (4): x <- x - (hbar_u^H x - sbar_u) hbar_u,
 *     and sbar carries the cluster index: sbar_{u,c} = p_{u,c} s_u.
 *
 * Pins (the CPU tests check these functions against what the paper and the mathematics fix, not
 * against themselves): the sweeps against Gauss-Seidel / dual Gauss-Seidel splittings and their
 * limits (local L-MMSE and local ZF by Cholesky), closed forms (one user, orthogonal columns, K = 0,
 * one cluster), exhaustive ML on tiny QPSK cases; the learned sweeps and fusion against hand-computed
 * values.  Parity unpinned: the COLNORM fusion weights' agreement with the paper's sigma_c^2, which
 * the paper does not state (only the reading above and its invariants are pinned: weights summing
 * to one, equal weights for identical clusters, the closed form for a scaled cluster).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double _Complex cplx;

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_ENOTPD (-3)

#define ORC_FUSE_EQUAL 0
#define ORC_FUSE_COLNORM 1

static double abs2(cplx z) { return creal(z) * creal(z) + cimag(z) * cimag(z); }

static int check_dims(int n_sc, int n_sym, int B, int U, int C, const int *csize, int f0, int f1)
{
    if (n_sc < 0 || n_sym < 1 || B < 1 || U < 1 || C < 1 || !csize) return ORC_EINVAL;
    if (f0 < 0 || f1 > n_sc || f0 > f1) return ORC_EINVAL;
    int sum = 0;
    for (int c = 0; c < C; ++c) {
        if (csize[c] < 1) return ORC_EINVAL;
        sum += csize[c];
    }
    return sum == B ? ORC_OK : ORC_EINVAL;
}

/*
 * Algorithm 1 (decentralized L-MMSE detection using CD), subcarriers f0 <= f < f1.
 *   Preprocessing: m_{u,c} = (||h_{u,c}||^2 + N0/Ex)^{-1},  n_{u,c} = m_{u,c} ||h_{u,c}||^2.
 *   Init r_c = y_c, x_c = 0.  For t = 1..K, for u = 1..U (cyclic, ascending):
 *       x_u <- m_{u,c} h_{u,c}^H r_c + n_{u,c} x_u;  dx = new - old;  r_c <- r_c - h_{u,c} dx.
 *   Fusion (Sec. III): xhat = sum_c lambda_c x_c, lambda_c = sigma_c^{-2} / sum_c' sigma_c'^{-2}.
 * fuse: ORC_FUSE_EQUAL (lambda_c = 1/C) or ORC_FUSE_COLNORM (sigma_c^2 reading above).
 * Xc and lam may be NULL.
 */
int oracle_detect(int n_sc, int n_sym, int B, int U, int C, const int *csize, int K, double Ex,
                  int fuse, const cplx *H, const cplx *Y, const double *N0, cplx *Xhat, cplx *Xc,
                  double *lam, int f0, int f1)
{
    if (check_dims(n_sc, n_sym, B, U, C, csize, f0, f1) != ORC_OK || K < 0 || !(Ex > 0)) return ORC_EINVAL;
    if (fuse != ORC_FUSE_EQUAL && fuse != ORC_FUSE_COLNORM) return ORC_EINVAL;
    if (!H || !Y || !N0 || !Xhat) return ORC_EINVAL;

    cplx *r = malloc(sizeof(cplx) * B);
    cplx *x = malloc(sizeof(cplx) * U);
    double *m = malloc(sizeof(double) * U);
    double *nn = malloc(sizeof(double) * U);
    double *w = malloc(sizeof(double) * C);
    double *lc = malloc(sizeof(double) * C);
    cplx *xc = malloc(sizeof(cplx) * (size_t)C * n_sym * U);
    int rc = ORC_OK;
    if (!r || !x || !m || !nn || !w || !lc || !xc) { rc = ORC_ENOMEM; goto out; }

    for (int f = f0; f < f1; ++f) {
        const double alpha = N0[f] / Ex;
        const cplx *Hf = H + (size_t)f * U * B;
        int o = 0;
        for (int c = 0; c < C; ++c) {
            const int Bc = csize[c];
            /* Preprocessing (decentralized). */
            double inv_sigma_sum = 0.0; /* sum_u (||h_u||^2 + alpha)^{-1}, up to the factor N0/U */
            for (int u = 0; u < U; ++u) {
                double e = 0.0;
                for (int b = 0; b < Bc; ++b) e += abs2(Hf[(size_t)u * B + o + b]);
                const double den = e + alpha;
                m[u] = den > 0.0 ? 1.0 / den : 0.0;
                nn[u] = m[u] * e;
                inv_sigma_sum += den > 0.0 ? 1.0 / den : INFINITY;
            }
            w[c] = 1.0 / inv_sigma_sum; /* proportional to sigma_c^{-2} */

            /* CD iterations (decentralized), independently per OFDM symbol. */
            for (int n = 0; n < n_sym; ++n) {
                const cplx *y = Y + ((size_t)f * n_sym + n) * B + o;
                for (int b = 0; b < Bc; ++b) r[b] = y[b];
                for (int u = 0; u < U; ++u) x[u] = 0.0;
                for (int t = 1; t <= K; ++t) {
                    for (int u = 0; u < U; ++u) {
                        const cplx *h = Hf + (size_t)u * B + o;
                        cplx corr = 0.0;
                        for (int b = 0; b < Bc; ++b) corr += conj(h[b]) * r[b];
                        const cplx xnew = m[u] * corr + nn[u] * x[u];
                        const cplx dx = xnew - x[u];
                        x[u] = xnew;
                        for (int b = 0; b < Bc; ++b) r[b] -= h[b] * dx;
                    }
                }
                for (int u = 0; u < U; ++u) xc[((size_t)c * n_sym + n) * U + u] = x[u];
            }
            o += Bc;
        }

        /* Data fusion (centralized). */
        double wsum = 0.0;
        for (int c = 0; c < C; ++c) wsum += w[c];
        for (int c = 0; c < C; ++c) {
            if (fuse == ORC_FUSE_EQUAL || !(wsum > 0.0))
                lc[c] = 1.0 / C;
            else
                lc[c] = w[c] / wsum;
            if (lam) lam[(size_t)f * C + c] = lc[c];
        }
        for (int n = 0; n < n_sym; ++n)
            for (int u = 0; u < U; ++u) {
                cplx acc = 0.0;
                for (int c = 0; c < C; ++c) acc += lc[c] * xc[((size_t)c * n_sym + n) * U + u];
                Xhat[((size_t)f * n_sym + n) * U + u] = acc;
            }
        if (Xc)
            memcpy(Xc + (size_t)f * C * n_sym * U, xc, sizeof(cplx) * (size_t)C * n_sym * U);
    }
out:
    free(r); free(x); free(m); free(nn); free(w); free(lc); free(xc);
    return rc;
}

/*
 * Algorithm 2 (decentralized ZF precoding using CD) with the per-cluster power normalization of
 * Sec. IV-B, subcarriers f0 <= f < f1.
 *   Preprocessing: p_{u,c} = ||h_{u,c}||^{-1}, hbar_{u,c} = p_{u,c} h_{u,c}, sbar_{u,c} = p_{u,c} s_u.
 *   Init x_c = 0.  For t = 1..K, for u = 1..U: x_c <- x_c - (hbar_{u,c}^H x_c - sbar_{u,c}) hbar_{u,c}
 *   (Eq. (4): the primal image of one coordinate step on the dual (2), Eq. (3)).
 *   Then x_c <- rho_c x_c / ||x_c||, rho_c = rho / sqrt(C); output [x_1; ...; x_C].
 */
int oracle_precode(int n_sc, int n_sym, int B, int U, int C, const int *csize, int K, double rho,
                   const cplx *H, const cplx *S, cplx *Xdl, int f0, int f1)
{
    if (check_dims(n_sc, n_sym, B, U, C, csize, f0, f1) != ORC_OK || K < 0) return ORC_EINVAL;
    if (!H || !S || !Xdl) return ORC_EINVAL;
    int Bmax = 0;
    for (int c = 0; c < C; ++c) Bmax = csize[c] > Bmax ? csize[c] : Bmax;
    cplx *hbar = malloc(sizeof(cplx) * (size_t)U * Bmax);
    double *p = malloc(sizeof(double) * U);
    cplx *sbar = malloc(sizeof(cplx) * U);
    cplx *x = malloc(sizeof(cplx) * Bmax);
    int rc = ORC_OK;
    if (!hbar || !p || !sbar || !x) { rc = ORC_ENOMEM; goto out; }
    const double rho_c = rho / sqrt((double)C);

    for (int f = f0; f < f1; ++f) {
        const cplx *Hf = H + (size_t)f * U * B;
        int o = 0;
        for (int c = 0; c < C; ++c) {
            const int Bc = csize[c];
            /* Preprocessing (decentralized): row-normalized local channel. */
            for (int u = 0; u < U; ++u) {
                double e = 0.0;
                for (int b = 0; b < Bc; ++b) e += abs2(Hf[(size_t)u * B + o + b]);
                p[u] = e > 0.0 ? 1.0 / sqrt(e) : 0.0;
                for (int b = 0; b < Bc; ++b) hbar[(size_t)u * Bc + b] = p[u] * Hf[(size_t)u * B + o + b];
            }
            for (int n = 0; n < n_sym; ++n) {
                const cplx *s = S + ((size_t)f * n_sym + n) * U;
                for (int u = 0; u < U; ++u) sbar[u] = p[u] * s[u];
                for (int b = 0; b < Bc; ++b) x[b] = 0.0;
                /* CD iterations (decentralized). */
                for (int t = 1; t <= K; ++t) {
                    for (int u = 0; u < U; ++u) {
                        const cplx *hb = hbar + (size_t)u * Bc;
                        cplx resid = 0.0;
                        for (int b = 0; b < Bc; ++b) resid += conj(hb[b]) * x[b];
                        resid -= sbar[u];
                        for (int b = 0; b < Bc; ++b) x[b] -= resid * hb[b];
                    }
                }
                /* Per-cluster power normalization (decentralized). */
                double nrm2 = 0.0;
                for (int b = 0; b < Bc; ++b) nrm2 += abs2(x[b]);
                const double nrm = sqrt(nrm2);
                cplx *out = Xdl + ((size_t)f * n_sym + n) * B + o;
                for (int b = 0; b < Bc; ++b) out[b] = nrm > 0.0 ? rho_c * x[b] / nrm : 0.0;
            }
            o += Bc;
        }
    }
out:
    free(hbar); free(p); free(sbar); free(x);
    return rc;
}

/* In-place Cholesky A = L L^H of an n x n Hermitian positive-definite matrix (row-major, lower
 * triangle of A overwritten by L).  Textbook column-by-column algorithm. */
static int cholesky(cplx *A, int n)
{
    for (int j = 0; j < n; ++j) {
        double d = creal(A[(size_t)j * n + j]);
        for (int k = 0; k < j; ++k) d -= abs2(A[(size_t)j * n + k]);
        if (!(d > 0.0)) return ORC_ENOTPD;
        const double ljj = sqrt(d);
        A[(size_t)j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            cplx s = A[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) s -= A[(size_t)i * n + k] * conj(A[(size_t)j * n + k]);
            A[(size_t)i * n + j] = s / ljj;
        }
    }
    return ORC_OK;
}

/* Solve (L L^H) x = b in place in b. */
static void chol_solve(const cplx *L, int n, cplx *b)
{
    for (int i = 0; i < n; ++i) {
        cplx s = b[i];
        for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * b[k];
        b[i] = s / creal(L[(size_t)i * n + i]);
    }
    for (int i = n - 1; i >= 0; --i) {
        cplx s = b[i];
        for (int k = i + 1; k < n; ++k) s -= conj(L[(size_t)k * n + i]) * b[k];
        b[i] = s / creal(L[(size_t)i * n + i]);
    }
}

/*
 * L-MMSE estimate of Eq. (1), xhat = (H^H H + (N0/Ex) I)^{-1} H^H y, by Cholesky, using antenna
 * rows row0 .. row0+nrows-1 of H (all B rows: the centralized detector; one cluster's rows: that
 * cluster's local L-MMSE, the fixed point of Algorithm 1 as K grows).  X: [n_sc][n_sym][U].
 */
int oracle_lmmse(int n_sc, int n_sym, int B, int U, int row0, int nrows, double Ex, const cplx *H,
                 const cplx *Y, const double *N0, cplx *X)
{
    if (n_sc < 0 || n_sym < 1 || U < 1 || row0 < 0 || nrows < 1 || row0 + nrows > B || !(Ex > 0)) return ORC_EINVAL;
    cplx *A = malloc(sizeof(cplx) * (size_t)U * U);
    cplx *z = malloc(sizeof(cplx) * U);
    int rc = ORC_OK;
    if (!A || !z) { rc = ORC_ENOMEM; goto out; }
    for (int f = 0; f < n_sc && rc == ORC_OK; ++f) {
        const cplx *Hf = H + (size_t)f * U * B + row0;
        const double alpha = N0[f] / Ex;
        for (int i = 0; i < U; ++i)
            for (int j = 0; j < U; ++j) {
                cplx g = 0.0;
                for (int b = 0; b < nrows; ++b) g += conj(Hf[(size_t)i * B + b]) * Hf[(size_t)j * B + b];
                A[(size_t)i * U + j] = g + (i == j ? alpha : 0.0);
            }
        rc = cholesky(A, U);
        if (rc != ORC_OK) break;
        for (int n = 0; n < n_sym; ++n) {
            const cplx *y = Y + ((size_t)f * n_sym + n) * B + row0;
            for (int i = 0; i < U; ++i) {
                cplx s = 0.0;
                for (int b = 0; b < nrows; ++b) s += conj(Hf[(size_t)i * B + b]) * y[b];
                z[i] = s;
            }
            chol_solve(A, U, z);
            memcpy(X + ((size_t)f * n_sym + n) * U, z, sizeof(cplx) * U);
        }
    }
out:
    free(A); free(z);
    return rc;
}

/*
 * Local ZF precoder, the closed form quoted in Sec. IV-A, xhat = H^H (H H^H)^{-1} s, for the downlink
 * channel of antenna rows row0 .. row0+nrows-1 (H^dl_c = (H^ul_c)^H, Sec. II-B), before any power
 * scaling.  Needs nrows >= U.  X: [n_sc][n_sym][nrows].
 */
int oracle_zf(int n_sc, int n_sym, int B, int U, int row0, int nrows, const cplx *H, const cplx *S, cplx *X)
{
    if (n_sc < 0 || n_sym < 1 || U < 1 || row0 < 0 || nrows < 1 || row0 + nrows > B) return ORC_EINVAL;
    cplx *A = malloc(sizeof(cplx) * (size_t)U * U);
    cplx *z = malloc(sizeof(cplx) * U);
    int rc = ORC_OK;
    if (!A || !z) { rc = ORC_ENOMEM; goto out; }
    for (int f = 0; f < n_sc && rc == ORC_OK; ++f) {
        const cplx *Hf = H + (size_t)f * U * B + row0;
        /* H^dl (H^dl)^H: entry (i, j) = h_i^H h_j. */
        for (int i = 0; i < U; ++i)
            for (int j = 0; j < U; ++j) {
                cplx g = 0.0;
                for (int b = 0; b < nrows; ++b) g += conj(Hf[(size_t)i * B + b]) * Hf[(size_t)j * B + b];
                A[(size_t)i * U + j] = g;
            }
        rc = cholesky(A, U);
        if (rc != ORC_OK) break;
        for (int n = 0; n < n_sym; ++n) {
            memcpy(z, S + ((size_t)f * n_sym + n) * U, sizeof(cplx) * U);
            chol_solve(A, U, z);
            cplx *x = X + ((size_t)f * n_sym + n) * nrows;
            for (int b = 0; b < nrows; ++b) {
                cplx s = 0.0;
                for (int u = 0; u < U; ++u) s += Hf[(size_t)u * B + b] * z[u];
                x[b] = s;
            }
        }
    }
out:
    free(A); free(z);
    return rc;
}

/*
 * Exhaustive maximum-likelihood detection, argmin over x in O^U of ||y - H x||^2, by enumerating all
 * M^U candidates (tiny problems only: the error-rate floor that any detector is compared with).
 * H: [n_vec][U][B] (row u = column h_u), Y: [n_vec][B], points: [M], labels: [n_vec][U].
 */
int oracle_ml(int n_vec, int B, int U, const cplx *H, const cplx *Y, int M, const cplx *points, int *labels)
{
    if (n_vec < 0 || B < 1 || U < 1 || M < 2 || !points || !labels) return ORC_EINVAL;
    double total = pow((double)M, (double)U);
    if (total > 1e7) return ORC_EINVAL;
    int *idx = malloc(sizeof(int) * U);
    int *best = malloc(sizeof(int) * U);
    cplx *e = malloc(sizeof(cplx) * B);
    int rc = ORC_OK;
    if (!idx || !best || !e) { rc = ORC_ENOMEM; goto out; }
    for (int v = 0; v < n_vec; ++v) {
        const cplx *Hv = H + (size_t)v * U * B;
        const cplx *y = Y + (size_t)v * B;
        double best_d = INFINITY;
        for (int u = 0; u < U; ++u) idx[u] = 0;
        for (;;) {
            double d = 0.0;
            for (int b = 0; b < B; ++b) {
                cplx s = y[b];
                for (int u = 0; u < U; ++u) s -= Hv[(size_t)u * B + b] * points[idx[u]];
                d += abs2(s);
            }
            if (d < best_d) {
                best_d = d;
                memcpy(best, idx, sizeof(int) * U);
            }
            int u = 0;
            while (u < U && ++idx[u] == M) idx[u++] = 0;
            if (u == U) break;
        }
        memcpy(labels + (size_t)v * U, best, sizeof(int) * U);
    }
out:
    free(idx); free(best); free(e);
    return rc;
}

/* ============================================================================================== */
/* Deep-unfolded CD with learned fusion (not in the paper: a learned extension of Algorithm 1).     */
/* ============================================================================================== */
/*
 * Parameters ("masters"): per sweep t, a step tau_t and a raw regularizer parameter gr_t with
 * gamma_t = softplus(gr_t) = log(1 + exp(gr_t)) > 0; a two-layer perceptron with hidden width Hd on
 * F = U + 1 per-cluster features phi_c = [||h_{1,c}||^2 / B_c, ..., ||h_{U,c}||^2 / B_c,
 * log10(max(N0/Ex, 1e-6))]: z = W1 phi + b1 (W1 row-major [Hd][F]), a = max(z, 0),
 * logit_c = w2 . a + b2, lambda = softmax_c(logit).
 *
 * Sweep t, user u (Gauss-Seidel order as in Algorithm 1), with e = ||h_{u,c}||^2, alpha = N0/Ex:
 *     x_u <- x_u + tau_t (h_u^H r - gamma_t alpha x_u) / (e + gamma_t alpha),   r <- r - h_u dx,
 * i.e. x_new = a1 g + a2 x_old with a1 = tau_t / (e + gamma_t alpha), a2 = 1 - tau_t gamma_t alpha /
 * (e + gamma_t alpha); tau_t = gamma_t = 1 is exactly Algorithm 1's update (a1 = m, a2 = n).  A
 * column with e + gamma_t alpha <= 0 is skipped (a1 = 0, a2 = 1).
 *
 * Loss: L = (1 / (n_sc n_sym)) sum_{f,n} ||xhat_{f,n} - xtarget_{f,n}||^2.
 */

static double softplus(double v) { return v > 30.0 ? v : log1p(exp(v)); }
static double sigmoid(double v) { return 1.0 / (1.0 + exp(-v)); }

typedef struct {
    int K, U, Hd, F;
    const double *tau, *graw, *W1, *b1, *w2;
    double b2;
} orc_learned;

/* Coefficients (a1, a2) of sweep t for a column of energy e. */
static void learned_coef(const orc_learned *P, int t, double e, double alpha, double *a1, double *a2, double *den_out)
{
    const double gam = softplus(P->graw[t]);
    const double den = e + gam * alpha;
    *den_out = den;
    if (den > 0.0) {
        *a1 = P->tau[t] / den;
        *a2 = 1.0 - P->tau[t] * gam * alpha / den;
    } else {
        *a1 = 0.0;
        *a2 = 1.0;
    }
}

/* MLP forward for one cluster's features: hidden pre-activations z[Hd] and the logit. */
static double mlp_forward(const orc_learned *P, const double *phi, double *z)
{
    double logit = P->b2;
    for (int k = 0; k < P->Hd; ++k) {
        double s = P->b1[k];
        for (int j = 0; j < P->F; ++j) s += P->W1[(size_t)k * P->F + j] * phi[j];
        z[k] = s;
        logit += P->w2[k] * (s > 0.0 ? s : 0.0);
    }
    return logit;
}

/*
 * Forward and (if grad != NULL) reverse pass for subcarriers f0 <= f < f1.
 * grad layout (masters): [tau(K), graw(K), W1(Hd*F), b1(Hd), w2(Hd), b2]; accumulated (+=).
 * loss accumulated (+=) if non-NULL.  Xhat, Xc, lam outputs optional.
 */
static int learned_pass(int n_sc, int n_sym, int B, int U, int C, const int *csize, double Ex, const orc_learned *P,
                        const cplx *H, const cplx *Y, const double *N0, const cplx *Xt, cplx *Xhat, cplx *Xc,
                        double *lam_out, double *loss, double *grad, int f0, int f1)
{
    const int K = P->K, Hd = P->Hd, F = P->F;
    const double inv_nvec = 1.0 / ((double)n_sc * n_sym);
    int Bmax = 0;
    for (int c = 0; c < C; ++c) Bmax = csize[c] > Bmax ? csize[c] : Bmax;
    cplx *r = malloc(sizeof(cplx) * Bmax);
    cplx *rb = malloc(sizeof(cplx) * Bmax);
    cplx *x = malloc(sizeof(cplx) * U);
    cplx *xb = malloc(sizeof(cplx) * U);
    cplx *xc = malloc(sizeof(cplx) * (size_t)C * n_sym * U);
    cplx *gsave = malloc(sizeof(cplx) * (size_t)K * U);   /* forward g per step (one tile) */
    cplx *xsave = malloc(sizeof(cplx) * (size_t)K * U);   /* forward x_old per step */
    double *e = malloc(sizeof(double) * (size_t)C * U);
    double *phi = malloc(sizeof(double) * (size_t)C * F);
    double *z = malloc(sizeof(double) * (size_t)C * Hd);
    double *logit = malloc(sizeof(double) * C);
    double *lam = malloc(sizeof(double) * C);
    double *lamb = malloc(sizeof(double) * C);
    double *a1b = malloc(sizeof(double) * (size_t)K * C * U); /* adjoints of a1, a2 per (t, c, u) */
    double *a2b = malloc(sizeof(double) * (size_t)K * C * U);
    cplx *gb = malloc(sizeof(cplx) * (size_t)n_sym * U);      /* dL/dxhat for this subcarrier */
    int rc = ORC_OK;
    if (!r || !rb || !x || !xb || !xc || !gsave || !xsave || !e || !phi || !z || !logit || !lam || !lamb || !a1b ||
        !a2b || !gb) {
        rc = ORC_ENOMEM;
        goto out;
    }
    for (int f = f0; f < f1; ++f) {
        const cplx *Hf = H + (size_t)f * U * B;
        const double alpha = N0[f] / Ex;
        /* features and fusion weights */
        int o = 0;
        for (int c = 0; c < C; ++c) {
            for (int u = 0; u < U; ++u) {
                double s = 0.0;
                for (int b = 0; b < csize[c]; ++b) s += abs2(Hf[(size_t)u * B + o + b]);
                e[c * U + u] = s;
                phi[c * F + u] = s / csize[c];
            }
            phi[c * F + U] = log10(alpha > 1e-6 ? alpha : 1e-6);
            logit[c] = mlp_forward(P, phi + c * F, z + (size_t)c * Hd);
            o += csize[c];
        }
        double mx = logit[0];
        for (int c = 1; c < C; ++c) mx = logit[c] > mx ? logit[c] : mx;
        double zs = 0.0;
        for (int c = 0; c < C; ++c) zs += exp(logit[c] - mx);
        for (int c = 0; c < C; ++c) {
            lam[c] = exp(logit[c] - mx) / zs;
            if (lam_out) lam_out[(size_t)f * C + c] = lam[c];
        }
        /* unfolded CD per cluster and symbol (forward) */
        o = 0;
        for (int c = 0; c < C; ++c) {
            const int Bc = csize[c];
            for (int n = 0; n < n_sym; ++n) {
                const cplx *y = Y + ((size_t)f * n_sym + n) * B + o;
                for (int b = 0; b < Bc; ++b) r[b] = y[b];
                for (int u = 0; u < U; ++u) x[u] = 0.0;
                for (int t = 0; t < K; ++t)
                    for (int u = 0; u < U; ++u) {
                        const cplx *h = Hf + (size_t)u * B + o;
                        double a1, a2, den;
                        learned_coef(P, t, e[c * U + u], alpha, &a1, &a2, &den);
                        cplx g = 0.0;
                        for (int b = 0; b < Bc; ++b) g += conj(h[b]) * r[b];
                        const cplx xn = a1 * g + a2 * x[u];
                        const cplx dx = xn - x[u];
                        x[u] = xn;
                        for (int b = 0; b < Bc; ++b) r[b] -= h[b] * dx;
                    }
                for (int u = 0; u < U; ++u) xc[((size_t)c * n_sym + n) * U + u] = x[u];
            }
            o += Bc;
        }
        for (int n = 0; n < n_sym; ++n)
            for (int u = 0; u < U; ++u) {
                cplx acc = 0.0;
                for (int c = 0; c < C; ++c) acc += lam[c] * xc[((size_t)c * n_sym + n) * U + u];
                if (Xhat) Xhat[((size_t)f * n_sym + n) * U + u] = acc;
                if (Xt) {
                    const cplx d = acc - Xt[((size_t)f * n_sym + n) * U + u];
                    if (loss) *loss += abs2(d) * inv_nvec;
                    gb[(size_t)n * U + u] = 2.0 * inv_nvec * d;
                }
            }
        if (Xc) memcpy(Xc + (size_t)f * C * n_sym * U, xc, sizeof(cplx) * (size_t)C * n_sym * U);
        if (!grad || !Xt) continue;

        /* ---- reverse pass ---- */
        double *g_tau = grad, *g_gr = grad + K, *g_W1 = grad + 2 * K, *g_b1 = g_W1 + (size_t)Hd * F;
        double *g_w2 = g_b1 + Hd, *g_b2 = g_w2 + Hd;
        /* fusion: xhat = sum_c lam_c x_c */
        double dot = 0.0;
        for (int c = 0; c < C; ++c) {
            double s = 0.0;
            for (int i = 0; i < n_sym * U; ++i) s += creal(conj(gb[i]) * xc[(size_t)c * n_sym * U + i]);
            lamb[c] = s;
            dot += lam[c] * s;
        }
        for (int c = 0; c < C; ++c) {
            const double lb = lam[c] * (lamb[c] - dot); /* softmax adjoint -> d logit_c */
            const double *zc = z + (size_t)c * Hd;
            *g_b2 += lb;
            for (int k = 0; k < Hd; ++k) {
                const double act = zc[k] > 0.0 ? zc[k] : 0.0;
                g_w2[k] += lb * act;
                const double zb = zc[k] > 0.0 ? lb * P->w2[k] : 0.0;
                g_b1[k] += zb;
                for (int j = 0; j < F; ++j) g_W1[(size_t)k * F + j] += zb * phi[c * F + j];
            }
        }
        /* unfolded CD: recompute each tile's forward steps, then walk them backwards */
        for (size_t i = 0; i < (size_t)K * C * U; ++i) a1b[i] = a2b[i] = 0.0;
        o = 0;
        for (int c = 0; c < C; ++c) {
            const int Bc = csize[c];
            for (int n = 0; n < n_sym; ++n) {
                const cplx *y = Y + ((size_t)f * n_sym + n) * B + o;
                for (int b = 0; b < Bc; ++b) r[b] = y[b];
                for (int u = 0; u < U; ++u) x[u] = 0.0;
                for (int t = 0; t < K; ++t)
                    for (int u = 0; u < U; ++u) {
                        const cplx *h = Hf + (size_t)u * B + o;
                        double a1, a2, den;
                        learned_coef(P, t, e[c * U + u], alpha, &a1, &a2, &den);
                        cplx g = 0.0;
                        for (int b = 0; b < Bc; ++b) g += conj(h[b]) * r[b];
                        gsave[(size_t)t * U + u] = g;
                        xsave[(size_t)t * U + u] = x[u];
                        const cplx xn = a1 * g + a2 * x[u];
                        const cplx dx = xn - x[u];
                        x[u] = xn;
                        for (int b = 0; b < Bc; ++b) r[b] -= h[b] * dx;
                    }
                for (int u = 0; u < U; ++u) xb[u] = lam[c] * gb[(size_t)n * U + u];
                for (int b = 0; b < Bc; ++b) rb[b] = 0.0;
                for (int t = K - 1; t >= 0; --t)
                    for (int u = U - 1; u >= 0; --u) {
                        const cplx *h = Hf + (size_t)u * B + o;
                        double a1, a2, den;
                        learned_coef(P, t, e[c * U + u], alpha, &a1, &a2, &den);
                        cplx hr = 0.0;
                        for (int b = 0; b < Bc; ++b) hr += conj(h[b]) * rb[b];
                        const cplx db = xb[u] - hr; /* adjoint of dx */
                        a1b[((size_t)t * C + c) * U + u] += creal(conj(db) * gsave[(size_t)t * U + u]);
                        a2b[((size_t)t * C + c) * U + u] += creal(conj(db) * xsave[(size_t)t * U + u]);
                        const cplx gbar = a1 * db;
                        for (int b = 0; b < Bc; ++b) rb[b] += h[b] * gbar;
                        xb[u] += (a2 - 1.0) * db;
                    }
            }
            o += Bc;
        }
        /* chain (a1, a2) -> (tau_t, gamma_t) -> raw parameter */
        for (int t = 0; t < K; ++t) {
            const double gam = softplus(P->graw[t]);
            double gt = 0.0, gg = 0.0;
            for (int c = 0; c < C; ++c)
                for (int u = 0; u < U; ++u) {
                    const double ev = e[c * U + u], den = ev + gam * alpha;
                    if (!(den > 0.0)) continue;
                    const double A1 = a1b[((size_t)t * C + c) * U + u], A2 = a2b[((size_t)t * C + c) * U + u];
                    gt += A1 / den - A2 * gam * alpha / den;
                    gg += -A1 * P->tau[t] * alpha / (den * den) - A2 * P->tau[t] * alpha * ev / (den * den);
                }
            g_tau[t] += gt;
            g_gr[t] += gg * sigmoid(P->graw[t]);
        }
    }
out:
    free(r); free(rb); free(x); free(xb); free(xc); free(gsave); free(xsave); free(e); free(phi); free(z);
    free(logit); free(lam); free(lamb); free(a1b); free(a2b); free(gb);
    return rc;
}

/* Public wrappers.  master: [tau(K), graw(K), W1(Hd*F), b1(Hd), w2(Hd), b2] with F = U + 1. */
static int learned_setup(orc_learned *P, int K, int U, int Hd, const double *master)
{
    if (K < 0 || U < 1 || Hd < 1 || !master) return ORC_EINVAL;
    P->K = K;
    P->U = U;
    P->Hd = Hd;
    P->F = U + 1;
    P->tau = master;
    P->graw = master + K;
    P->W1 = master + 2 * K;
    P->b1 = P->W1 + (size_t)Hd * P->F;
    P->w2 = P->b1 + Hd;
    P->b2 = P->w2[Hd];
    return ORC_OK;
}

int oracle_learned_forward(int n_sc, int n_sym, int B, int U, int C, const int *csize, int K, double Ex, int Hd,
                           const double *master, const cplx *H, const cplx *Y, const double *N0, cplx *Xhat, cplx *Xc,
                           double *lam, int f0, int f1)
{
    orc_learned P;
    if (check_dims(n_sc, n_sym, B, U, C, csize, f0, f1) != ORC_OK || !(Ex > 0)) return ORC_EINVAL;
    if (learned_setup(&P, K, U, Hd, master) != ORC_OK || !H || !Y || !N0) return ORC_EINVAL;
    return learned_pass(n_sc, n_sym, B, U, C, csize, Ex, &P, H, Y, N0, NULL, Xhat, Xc, lam, NULL, NULL, f0, f1);
}

/* Loss and gradient (accumulated into grad[] and *loss, which the caller zeroes). */
int oracle_learned_grad(int n_sc, int n_sym, int B, int U, int C, const int *csize, int K, double Ex, int Hd,
                        const double *master, const cplx *H, const cplx *Y, const double *N0, const cplx *Xt,
                        double *loss, double *grad, int f0, int f1)
{
    orc_learned P;
    if (check_dims(n_sc, n_sym, B, U, C, csize, f0, f1) != ORC_OK || !(Ex > 0)) return ORC_EINVAL;
    if (learned_setup(&P, K, U, Hd, master) != ORC_OK || !H || !Y || !N0 || !Xt || !loss || !grad) return ORC_EINVAL;
    return learned_pass(n_sc, n_sym, B, U, C, csize, Ex, &P, H, Y, N0, Xt, NULL, NULL, NULL, loss, grad, f0, f1);
}
