/*
 * Plain FP64 oracle: Galerkin integrals of the Maxwell boundary operators S
 * and C on pairs of flat triangles.  TEST INFRASTRUCTURE ONLY — called from
 * oracle/bem.py, never linked into the CUDA library.
 *
 * Paper (arXiv 2008.04772), Section 2: G(x,y) = e^{ik|x-y|} / (4 pi |x-y|),
 * S = gamma_D E, C = gamma_D H with gamma_D P = P x n, tested with the pairing
 * <a,b> = int a . (n x b) (eq. dualpairingGammam). For tangential div-conforming
 * trial/test functions phi_j, phi_i on a closed surface this gives
 *
 *   <S phi_j, phi_i> = -ik  II G phi_i(x).phi_j(y)
 *                      + (i/k) II G div phi_i(x) div phi_j(y)
 *   <C phi_j, phi_i> =  II grad_x G(x,y) . (phi_i(x) x phi_j(y)),
 *   grad_x G = (x-y) (ik r - 1) e^{ikr} / (4 pi r^3).
 *
 * Local functions on triangle tau with vertices P_0..P_2:
 * f_a(x) = (x - P_a) / (2|tau|), div f_a = 1/|tau|.
 *
 * Quadrature (Section 3.3): disjoint closures -> tensor product of a symmetric
 * triangle rule, chosen by the pair's near / medium / far class (relative
 * distance |c1 - c2| / max(d1, d2) of centroids and longest edges, against
 * the bounds b_near, b_med); shared vertex / edge / identical -> Sauter–Schwab rules on
 * [0,1]^4 (2 / 5 / 6 sub-regions, Gauss–Legendre in each coordinate).  The
 * integrand is evaluated directly from the formulas above — no moment algebra.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

typedef struct {
    double P[3][3];  /* vertices in storage order */
    double A;        /* area */
} tri_t;

static void sub3(const double *a, const double *b, double *c) {
    c[0] = a[0] - b[0]; c[1] = a[1] - b[1]; c[2] = a[2] - b[2];
}
static double dot3(const double *a, const double *b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static void cross3(const double *a, const double *b, double *c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static void load_tri(const double *X, const long *ids, long t, tri_t *T) {
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) T->P[a][c] = X[3 * ids[3 * t + a] + c];
    double u[3], v[3], n[3];
    sub3(T->P[1], T->P[0], u);
    sub3(T->P[2], T->P[0], v);
    cross3(u, v, n);
    T->A = 0.5 * sqrt(dot3(n, n));
}

/* one quadrature point pair (x on t1, y on t2, weight w) added to both blocks */
static void add_point_pair(const tri_t *t1, const tri_t *t2, const double *x,
                           const double *y, double w, cplx k, int want,
                           cplx *S, cplx *C) {
    double d[3];
    sub3(x, y, d);
    double r = sqrt(dot3(d, d));
    cplx e = cexp(I * k * r);
    cplx G = e / (4.0 * M_PI * r);
    cplx gfac = (I * k * r - 1.0) * e / (4.0 * M_PI * r * r * r);
    double fa[3][3], gb[3][3];
    for (int a = 0; a < 3; ++a) {
        double u[3];
        sub3(x, t1->P[a], u);
        for (int c = 0; c < 3; ++c) fa[a][c] = u[c] / (2.0 * t1->A);
        sub3(y, t2->P[a], u);
        for (int c = 0; c < 3; ++c) gb[a][c] = u[c] / (2.0 * t2->A);
    }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            if (want & 1)
                S[3 * a + b] += w * (-I * k * G * dot3(fa[a], gb[b]) +
                                     (I / k) * G / (t1->A * t2->A));
            if (want & 2) {
                double c[3];
                cross3(fa[a], gb[b], c);
                C[3 * a + b] += w * gfac * dot3(d, c);
            }
        }
}

/* Sauter–Schwab maps of [0,1]^4 onto pairs of reference triangles
 * {0 <= s2 <= s1 <= 1}; cls 1 = common vertex (reference point (0,0)),
 * cls 2 = common edge ((0,0)-(1,0)), cls 3 = identical.  Returns the number
 * of sub-regions; fills the reference points and the Jacobian of region r. */
static int ss_regions(int cls) { return cls == 3 ? 6 : (cls == 2 ? 5 : 2); }

static void ss_map(int cls, int r, double xi, double e1, double e2, double e3,
                   double *xh, double *yh, double *jac) {
    if (cls == 3) {
        *jac = xi * xi * xi * e1 * e1 * e2;
        switch (r) {
        case 0: xh[0] = xi; xh[1] = xi * (1 - e1 + e1 * e2);
                yh[0] = xi * (1 - e1 * e2 * e3); yh[1] = xi * (1 - e1); break;
        case 1: xh[0] = xi * (1 - e1 * e2 * e3); xh[1] = xi * (1 - e1);
                yh[0] = xi; yh[1] = xi * (1 - e1 + e1 * e2); break;
        case 2: xh[0] = xi; xh[1] = xi * e1 * (1 - e2 + e2 * e3);
                yh[0] = xi * (1 - e1 * e2); yh[1] = xi * e1 * (1 - e2); break;
        case 3: xh[0] = xi * (1 - e1 * e2); xh[1] = xi * e1 * (1 - e2);
                yh[0] = xi; yh[1] = xi * e1 * (1 - e2 + e2 * e3); break;
        case 4: xh[0] = xi * (1 - e1 * e2 * e3); xh[1] = xi * e1 * (1 - e2 * e3);
                yh[0] = xi; yh[1] = xi * e1 * (1 - e2); break;
        default: xh[0] = xi; xh[1] = xi * e1 * (1 - e2);
                 yh[0] = xi * (1 - e1 * e2 * e3); yh[1] = xi * e1 * (1 - e2 * e3); break;
        }
    } else if (cls == 2) {
        *jac = xi * xi * xi * e1 * e1 * (r == 0 ? 1.0 : e2);
        switch (r) {
        case 0: xh[0] = xi; xh[1] = xi * e1 * e3;
                yh[0] = xi * (1 - e1 * e2); yh[1] = xi * e1 * (1 - e2); break;
        case 1: xh[0] = xi; xh[1] = xi * e1;
                yh[0] = xi * (1 - e1 * e2 * e3); yh[1] = xi * e1 * e2 * (1 - e3); break;
        case 2: xh[0] = xi * (1 - e1 * e2); xh[1] = xi * e1 * (1 - e2);
                yh[0] = xi; yh[1] = xi * e1 * e2 * e3; break;
        case 3: xh[0] = xi * (1 - e1 * e2 * e3); xh[1] = xi * e1 * e2 * (1 - e3);
                yh[0] = xi; yh[1] = xi * e1; break;
        default: xh[0] = xi * (1 - e1 * e2 * e3); xh[1] = xi * e1 * (1 - e2 * e3);
                 yh[0] = xi; yh[1] = xi * e1 * e2; break;
        }
    } else {
        *jac = xi * xi * xi * e2;
        if (r == 0) { xh[0] = xi; xh[1] = xi * e1; yh[0] = xi * e2; yh[1] = xi * e2 * e3; }
        else        { xh[0] = xi * e2; xh[1] = xi * e2 * e3; yh[0] = xi; yh[1] = xi * e1; }
    }
}

/* reference point (s1, s2) -> Q0 + s1 (Q1 - Q0) + s2 (Q2 - Q1) */
static void ref_to_phys(const double Q[3][3], const double *s, double *x) {
    for (int c = 0; c < 3; ++c)
        x[c] = Q[0][c] + s[0] * (Q[1][c] - Q[0][c]) + s[1] * (Q[2][c] - Q[1][c]);
}

/* Number of shared vertex ids and the canonical parametrisation orders:
 * shared vertices first, in the same order on both triangles. */
static int classify(const long *i1, const long *i2, int o1[3], int o2[3]) {
    int s1[3], s2[3], ns = 0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            if (i1[a] == i2[b]) { s1[ns] = a; s2[ns] = b; ++ns; }
    if (ns == 0) return 0;
    if (ns == 3) {
        for (int a = 0; a < 3; ++a) { o1[a] = a; o2[a] = s2[a]; }
        /* o2[a] must be the trial local index of the same vertex as o1[a] */
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                if (i2[b] == i1[a]) o2[a] = b;
        return 3;
    }
    for (int q = 0; q < ns; ++q) { o1[q] = s1[q]; o2[q] = s2[q]; }
    /* fill the remaining local indices in storage order */
    int n1 = ns, n2 = ns;
    for (int a = 0; a < 3; ++a) {
        int used1 = 0, used2 = 0;
        for (int q = 0; q < ns; ++q) { used1 |= (s1[q] == a); used2 |= (s2[q] == a); }
        if (!used1) o1[n1++] = a;
        if (!used2) o2[n2++] = a;
    }
    return ns;
}

/*
 * Local blocks for test triangles test[0..n1) x trial triangles trial[0..n2).
 * S, C: [n1][n2][3][3] complex (interleaved doubles); want bit 1 = S, 2 = C.
 * counts[0..3]: integrand evaluations for regular / vertex / edge / identical pairs.
 */
/* centroid and longest edge of a triangle */
static void tri_size(const tri_t *t, double *c, double *d) {
    double l = 0.0;
    for (int a = 0; a < 3; ++a) {
        double e[3];
        sub3(t->P[(a + 1) % 3], t->P[a], e);
        const double q = sqrt(dot3(e, e));
        if (q > l) l = q;
    }
    for (int k = 0; k < 3; ++k) c[k] = (t->P[0][k] + t->P[1][k] + t->P[2][k]) / 3.0;
    *d = l;
}

/* class of a regular pair: 0 near, 1 medium, 2 far */
static int regular_class(const tri_t *t1, const tri_t *t2, double b_near, double b_med) {
    double c1[3], c2[3], d1, d2, dc[3];
    tri_size(t1, c1, &d1);
    tri_size(t2, c2, &d2);
    sub3(c1, c2, dc);
    const double rel = sqrt(dot3(dc, dc)) / (d1 > d2 ? d1 : d2);
    return rel <= b_near ? 0 : (rel <= b_med ? 1 : 2);
}

/* npts[3], rbary (3 npts[c] per class, concatenated), rw (npts[c] per class):
 * the near / medium / far rules; the same rule three times for one rule. */
void orc_blocks(const double *X, const long *ids, const long *test, long n1,
                const long *trial, long n2, double kr, double ki, int want,
                const int *npts, const double *rbary_all, const double *rw_all, double b_near,
                double b_med, int ng, const double *gx, const double *gw, double *Sout,
                double *Cout, long *counts) {
    cplx k = kr + I * ki;
    long cnt[4] = {0, 0, 0, 0};
#pragma omp parallel
    {
        long lc[4] = {0, 0, 0, 0};
#pragma omp for schedule(dynamic, 1)
        for (long p = 0; p < n1; ++p) {
            tri_t t1;
            load_tri(X, ids, test[p], &t1);
            const long *i1 = ids + 3 * test[p];
            for (long q = 0; q < n2; ++q) {
                tri_t t2;
                load_tri(X, ids, trial[q], &t2);
                const long *i2 = ids + 3 * trial[q];
                cplx S[9], C[9];
                for (int m = 0; m < 9; ++m) { S[m] = 0; C[m] = 0; }
                int o1[3], o2[3];
                int cls = classify(i1, i2, o1, o2);
                if (cls == 0) {
                    const int rc = regular_class(&t1, &t2, b_near, b_med);
                    int off = 0;
                    for (int c = 0; c < rc; ++c) off += npts[c];
                    const int nreg = npts[rc];
                    const double *rbary = rbary_all + 3 * off, *rw = rw_all + off;
                    for (int u = 0; u < nreg; ++u) {
                        double x[3], y[3];
                        for (int c = 0; c < 3; ++c)
                            x[c] = rbary[3 * u] * t1.P[0][c] + rbary[3 * u + 1] * t1.P[1][c] +
                                   rbary[3 * u + 2] * t1.P[2][c];
                        for (int v = 0; v < nreg; ++v) {
                            for (int c = 0; c < 3; ++c)
                                y[c] = rbary[3 * v] * t2.P[0][c] + rbary[3 * v + 1] * t2.P[1][c] +
                                       rbary[3 * v + 2] * t2.P[2][c];
                            add_point_pair(&t1, &t2, x, y, rw[u] * t1.A * rw[v] * t2.A, k, want, S, C);
                            ++lc[0];
                        }
                    }
                } else {
                    double Q1[3][3], Q2[3][3];
                    for (int a = 0; a < 3; ++a)
                        for (int c = 0; c < 3; ++c) {
                            Q1[a][c] = t1.P[o1[a]][c];
                            Q2[a][c] = t2.P[o2[a]][c];
                        }
                    int nr = ss_regions(cls);
                    double scale = (2.0 * t1.A) * (2.0 * t2.A);
                    for (int r = 0; r < nr; ++r)
                        for (int a0 = 0; a0 < ng; ++a0)
                            for (int a1 = 0; a1 < ng; ++a1)
                                for (int a2 = 0; a2 < ng; ++a2)
                                    for (int a3 = 0; a3 < ng; ++a3) {
                                        double xh[2], yh[2], jac, x[3], y[3];
                                        ss_map(cls, r, gx[a0], gx[a1], gx[a2], gx[a3], xh, yh, &jac);
                                        ref_to_phys(Q1, xh, x);
                                        ref_to_phys(Q2, yh, y);
                                        double w = gw[a0] * gw[a1] * gw[a2] * gw[a3] * jac * scale;
                                        add_point_pair(&t1, &t2, x, y, w, k, want, S, C);
                                        ++lc[cls];
                                    }
                }
                double *so = Sout + 18 * (p * n2 + q);
                double *co = Cout + 18 * (p * n2 + q);
                for (int m = 0; m < 9; ++m) {
                    so[2 * m] = creal(S[m]); so[2 * m + 1] = cimag(S[m]);
                    co[2 * m] = creal(C[m]); co[2 * m + 1] = cimag(C[m]);
                }
            }
        }
#pragma omp critical
        for (int m = 0; m < 4; ++m) cnt[m] += lc[m];
    }
    if (counts)
        for (int m = 0; m < 4; ++m) counts[m] = cnt[m];
}

/*
 * Integral of a user-chosen smooth test kernel over a singular pair by the
 * same Sauter–Schwab machinery (used only to pin the maps): the kernel is the
 * polynomial  prod_c (1 + x_c)^px[c] * (1 + y_c)^py[c]  in physical coordinates.
 */
double orc_ss_polynomial(const double *P1, const double *P2, int cls, const int *o1,
                         const int *o2, const int *px, const int *py, int ng,
                         const double *gx, const double *gw) {
    double Q1[3][3], Q2[3][3], A1, A2, u[3], v[3], n[3];
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) {
            Q1[a][c] = P1[3 * o1[a] + c];
            Q2[a][c] = P2[3 * o2[a] + c];
        }
    sub3(P1 + 3, P1, u); sub3(P1 + 6, P1, v); cross3(u, v, n); A1 = 0.5 * sqrt(dot3(n, n));
    sub3(P2 + 3, P2, u); sub3(P2 + 6, P2, v); cross3(u, v, n); A2 = 0.5 * sqrt(dot3(n, n));
    double acc = 0.0;
    int nr = ss_regions(cls);
    for (int r = 0; r < nr; ++r)
        for (int a0 = 0; a0 < ng; ++a0)
            for (int a1 = 0; a1 < ng; ++a1)
                for (int a2 = 0; a2 < ng; ++a2)
                    for (int a3 = 0; a3 < ng; ++a3) {
                        double xh[2], yh[2], jac, x[3], y[3];
                        ss_map(cls, r, gx[a0], gx[a1], gx[a2], gx[a3], xh, yh, &jac);
                        ref_to_phys(Q1, xh, x);
                        ref_to_phys(Q2, yh, y);
                        double f = 1.0;
                        for (int c = 0; c < 3; ++c) f *= pow(1 + x[c], px[c]) * pow(1 + y[c], py[c]);
                        acc += gw[a0] * gw[a1] * gw[a2] * gw[a3] * jac * f;
                    }
    return acc * 4.0 * A1 * A2;
}
