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
