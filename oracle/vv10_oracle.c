/*
 * VV10 oracle: plain, slow, FP64 CPU restatement of the VV10 quadrature sums.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU
 * baseline may load this library.  It shares no code, header, table or constant with
 * the CUDA library, and the CUDA library never calls it.
 *
 * Every function follows the paper (Liang, Feng, Liu, Head-Gordon, arXiv 2208.14639,
 * Sec. II) term by term, in its notation:
 *   E      = sum_i w_i rho_i (beta + 1/2 E_i)                       (Sec. II.A, E^VV10 on a grid)
 *   E_i    = sum_j w_j rho_j Phi_ij                                 (Sec. II.A)
 *   Phi_ij = -3 / (2 g g' (g + g')),  g = omega_i R^2 + kappa_i,
 *            g' = omega_j R^2 + kappa_j                             (Eqs. Cknernal, g)
 *   omega  = sqrt(C gamma^2/rho^4 + 4 pi rho/3),
 *   kappa  = b (3 pi/2) (rho/(9 pi))^(1/6),
 *   beta   = (1/32) (3/b^2)^(3/4)                                   (Sec. II.A)
 *   f^rho_i, f^gamma_i, U_i, W_i                                    (Sec. II.A, Fock matrix)
 *   f^{rho,t}, f^{gamma,t} with f^{rho rho}, f^{gamma rho}, f^{rho gamma},
 *   f^{gamma gamma} and A_i, B_i, C_i                               (Sec. II.B, Eq. frhot)
 *   E^A_gr (first, unsimplified form) and E/U/W_i^{Bgr}             (Eqs. grad_gr, EiBgr)
 *   D_i^B and E^{AB}_{gr,gr}; E/U/W_i^{Bw} for given weight directions (Sec. II.B)
 *
 * Readings where the paper is silent:
 *   - the inner sums over j include j = i (Phi_ii = -3/(4 kappa_i^3) is finite, and the
 *     delta_ij/w_i terms of the second derivatives are then the exact Hessian);
 *   - points with rho < rho_cut are dropped from every sum and get zero outputs;
 *   - of the two printed forms of E^A_gr only the first is used (the second, simplified
 *     one disagrees with finite differences of E).
 *
 * All row sums and totals use Neumaier-compensated summation; rows run in parallel
 * (OpenMP), each row's sum is sequential over j in index order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* ---------------------------------------------------------------- compensated sums */
typedef struct { double s, c; } nsum;

static inline void nsum_add(nsum* a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static inline double nsum_get(const nsum* a) { return a->s + a->c; }

/* ---------------------------------------------------------------- point quantities */
typedef struct {
    double rho, gamma;
    double omega, kappa;
    double om_r, om_g;               /* d omega / d rho, d omega / d gamma         */
    double ka_r;                     /* d kappa / d rho                             */
    double om_rr, om_rg, om_gg;      /* second derivatives of omega                 */
    double ka_rr;                    /* d^2 kappa / d rho^2                         */
} orc_point;

double orc_beta(double b) { return pow(3.0 / (b * b), 0.75) / 32.0; }

/* omega, kappa and their derivatives at one point (Sec. II.A definitions).
 * Derivatives are taken of Q = omega^2 = C gamma^2 rho^-4 + 4 pi rho / 3:
 *   omega_x = Q_x / (2 omega),  omega_xy = Q_xy / (2 omega) - Q_x Q_y / (4 omega^3). */
static orc_point orc_point_eval(double rho, double gamma, double b, double C) {
    orc_point p;
    p.rho = rho;
    p.gamma = gamma;
    double r2 = rho * rho, r4 = r2 * r2;
    double Q = C * gamma * gamma / r4 + 4.0 * ORC_PI * rho / 3.0;
    double Qr = -4.0 * C * gamma * gamma / (r4 * rho) + 4.0 * ORC_PI / 3.0;
    double Qg = 2.0 * C * gamma / r4;
    double Qrr = 20.0 * C * gamma * gamma / (r4 * r2);
    double Qrg = -8.0 * C * gamma / (r4 * rho);
    double Qgg = 2.0 * C / r4;
    double om = sqrt(Q);
    p.omega = om;
    p.om_r = Qr / (2.0 * om);
    p.om_g = Qg / (2.0 * om);
    p.om_rr = Qrr / (2.0 * om) - Qr * Qr / (4.0 * om * om * om);
    p.om_rg = Qrg / (2.0 * om) - Qr * Qg / (4.0 * om * om * om);
    p.om_gg = Qgg / (2.0 * om) - Qg * Qg / (4.0 * om * om * om);
    p.kappa = b * 1.5 * ORC_PI * pow(rho / (9.0 * ORC_PI), 1.0 / 6.0);
    p.ka_r = p.kappa / (6.0 * rho);
    p.ka_rr = -5.0 * p.kappa / (36.0 * rho * rho);
    return p;
}

void orc_point_props(int64_t n, const double* rho, const double* grad, double b, double C,
                     double* out /* n x 11 */) {
    for (int64_t i = 0; i < n; ++i) {
        double gam = grad[3 * i] * grad[3 * i] + grad[3 * i + 1] * grad[3 * i + 1] +
                     grad[3 * i + 2] * grad[3 * i + 2];
        orc_point p = orc_point_eval(rho[i], gam, b, C);
        double* o = out + 11 * i;
        o[0] = p.gamma; o[1] = p.omega; o[2] = p.kappa; o[3] = p.om_r; o[4] = p.om_g;
        o[5] = p.ka_r; o[6] = p.om_rr; o[7] = p.om_rg; o[8] = p.om_gg; o[9] = p.ka_rr;
        o[10] = 0.0;
    }
}

/* Phi_ij for given endpoint quantities and squared distance (Eqs. Cknernal, g). */
double orc_phi(double om_i, double ka_i, double om_j, double ka_j, double R2) {
    double g = om_i * R2 + ka_i;
    double gp = om_j * R2 + ka_j;
    return -3.0 / (2.0 * g * gp * (g + gp));
}

/* ---------------------------------------------------------------- prepared system */
typedef struct {
    int64_t n;          /* all points                                  */
    int64_t nk;         /* kept points (rho >= rho_cut)                */
    int64_t* kept;      /* kept -> original index                      */
    int64_t* slot;      /* original -> kept index, or -1               */
    orc_point* pt;      /* per kept point                              */
    double* xyz;        /* per kept point, 3                           */
    double* w;          /* per kept point                              */
    double* grad;       /* per kept point, 3                           */
    double beta;
} orc_sys;

static void orc_sys_free(orc_sys* s) {
    free(s->kept); free(s->slot); free(s->pt); free(s->xyz); free(s->w); free(s->grad);
}

static int orc_sys_init(orc_sys* s, int64_t n, const double* xyz, const double* w,
                        const double* rho, const double* grad, double b, double C,
                        double rho_cut) {
    memset(s, 0, sizeof(*s));
    s->n = n;
    s->beta = orc_beta(b);
    s->kept = (int64_t*)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    s->slot = (int64_t*)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    s->pt = (orc_point*)malloc(sizeof(orc_point) * (n > 0 ? n : 1));
    s->xyz = (double*)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    s->w = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
    s->grad = (double*)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    if (!s->kept || !s->slot || !s->pt || !s->xyz || !s->w || !s->grad) {
        orc_sys_free(s);
        return -1;
    }
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!(rho[i] >= rho_cut)) { s->slot[i] = -1; continue; }
        double gam = grad[3 * i] * grad[3 * i] + grad[3 * i + 1] * grad[3 * i + 1] +
                     grad[3 * i + 2] * grad[3 * i + 2];
        s->slot[i] = k;
        s->kept[k] = i;
        s->pt[k] = orc_point_eval(rho[i], gam, b, C);
        for (int d = 0; d < 3; ++d) {
            s->xyz[3 * k + d] = xyz[3 * i + d];
            s->grad[3 * k + d] = grad[3 * i + d];
        }
        s->w[k] = w[i];
        ++k;
    }
    s->nk = k;
    return 0;
}

static inline double orc_r2(const orc_sys* s, int64_t a, int64_t c) {
    double dx = s->xyz[3 * a] - s->xyz[3 * c];
    double dy = s->xyz[3 * a + 1] - s->xyz[3 * c + 1];
    double dz = s->xyz[3 * a + 2] - s->xyz[3 * c + 2];
    return dx * dx + dy * dy + dz * dz;
}

/* ---------------------------------------------------------------- energy */
/* E^VV10 = sum_i w_i rho_i (beta + 1/2 sum_j w_j rho_j Phi_ij), straight from the
 * quadrature form of Eq. EVV10. */
int orc_energy(int64_t n, const double* xyz, const double* w, const double* rho,
               const double* grad, double b, double C, double rho_cut, double* energy) {
    orc_sys s;
    if (orc_sys_init(&s, n, xyz, w, rho, grad, b, C, rho_cut)) return -1;
    int64_t nk = s.nk;
    double* fi = (double*)malloc(sizeof(double) * (nk > 0 ? nk : 1));
    if (!fi) { orc_sys_free(&s); return -1; }
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t i = 0; i < nk; ++i) {
        nsum Ei = {0, 0};
        for (int64_t j = 0; j < nk; ++j) {
            double phi = orc_phi(s.pt[i].omega, s.pt[i].kappa, s.pt[j].omega, s.pt[j].kappa,
                                 orc_r2(&s, i, j));
            nsum_add(&Ei, s.w[j] * s.pt[j].rho * phi);
        }
        fi[i] = s.w[i] * s.pt[i].rho * (s.beta + 0.5 * nsum_get(&Ei));
    }
    nsum tot = {0, 0};
    for (int64_t i = 0; i < nk; ++i) nsum_add(&tot, fi[i]);
    *energy = nsum_get(&tot);
    free(fi);
    orc_sys_free(&s);
    return 0;
}

/* ---------------------------------------------------------------- pair sums */
/* Row sums E_i, U_i, W_i (Sec. II.A) and A_i, B_i, C_i (Sec. II.B) for one kept row. */
static void orc_row_sums(const orc_sys* s, int64_t i, double out[6]) {
    nsum E = {0, 0}, U = {0, 0}, W = {0, 0}, A = {0, 0}, B = {0, 0}, Cc = {0, 0};
    const orc_point* pi = &s->pt[i];
    for (int64_t j = 0; j < s->nk; ++j) {
        const orc_point* pj = &s->pt[j];
        double R2 = orc_r2(s, i, j);
        double g = pi->omega * R2 + pi->kappa;
        double gp = pj->omega * R2 + pj->kappa;
        double sg = g + gp;
        double phi = -3.0 / (2.0 * g * gp * sg);
        double cj = s->w[j] * pj->rho;
        double t1 = 1.0 / sg + 1.0 / g;
        double t2 = 1.0 / (sg * sg) + 1.0 / (sg * g) + 1.0 / (g * g);
        nsum_add(&E, cj * phi);
        nsum_add(&U, -cj * phi * t1);
        nsum_add(&W, -cj * phi * R2 * t1);
        nsum_add(&A, 2.0 * cj * phi * t2);
        nsum_add(&B, 2.0 * cj * phi * R2 * t2);
        nsum_add(&Cc, 2.0 * cj * phi * R2 * R2 * t2);
    }
    out[0] = nsum_get(&E); out[1] = nsum_get(&U); out[2] = nsum_get(&W);
    out[3] = nsum_get(&A); out[4] = nsum_get(&B); out[5] = nsum_get(&Cc);
}

/* rows: original indices (NULL = all n points).  out: n_rows x 6, {E,U,W,A,B,C};
 * rows that were dropped by the cutoff get zeros. */
int orc_pair_sums(int64_t n, const double* xyz, const double* w, const double* rho,
                  const double* grad, double b, double C, double rho_cut, int64_t n_rows,
                  const int64_t* rows, double* out) {
    orc_sys s;
    if (orc_sys_init(&s, n, xyz, w, rho, grad, b, C, rho_cut)) return -1;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t r = 0; r < n_rows; ++r) {
        int64_t i = rows ? rows[r] : r;
        int64_t k = s.slot[i];
        if (k < 0) { for (int q = 0; q < 6; ++q) out[6 * r + q] = 0.0; continue; }
        orc_row_sums(&s, k, out + 6 * r);
    }
    orc_sys_free(&s);
    return 0;
}

/* ---------------------------------------------------------------- potential */
/* f^rho_i = beta + E_i + rho_i (kappa'_i U_i + omega_rho,i W_i),
 * f^gamma_i = rho_i omega_gamma,i W_i                                   (Sec. II.A)
 * Also returns E (the energy) when `energy` is non-NULL and rows == NULL. */
int orc_potential(int64_t n, const double* xyz, const double* w, const double* rho,
                  const double* grad, double b, double C, double rho_cut, int64_t n_rows,
                  const int64_t* rows, double* vrho, double* vgamma, double* energy) {
    orc_sys s;
    if (orc_sys_init(&s, n, xyz, w, rho, grad, b, C, rho_cut)) return -1;
    double* fi = (double*)calloc((size_t)(n_rows > 0 ? n_rows : 1), sizeof(double));
    if (!fi) { orc_sys_free(&s); return -1; }
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t r = 0; r < n_rows; ++r) {
        int64_t i = rows ? rows[r] : r;
        int64_t k = s.slot[i];
        if (k < 0) { vrho[r] = 0.0; vgamma[r] = 0.0; fi[r] = 0.0; continue; }
        double sums[6];
        orc_row_sums(&s, k, sums);
        const orc_point* p = &s.pt[k];
        vrho[r] = s.beta + sums[0] + p->rho * (p->ka_r * sums[1] + p->om_r * sums[2]);
        vgamma[r] = p->rho * p->om_g * sums[2];
        fi[r] = s.w[k] * p->rho * (s.beta + 0.5 * sums[0]);
    }
    if (energy) {
        nsum tot = {0, 0};
        for (int64_t r = 0; r < n_rows; ++r) nsum_add(&tot, fi[r]);
        *energy = nsum_get(&tot);
    }
    free(fi);
    orc_sys_free(&s);
    return 0;
}

/* ---------------------------------------------------------------- Hessian contraction */
/* f^{rho,t}_i   = sum_j w_j (f^{rho rho}_ij rho^t_j + 2 f^{rho gamma}_ij gamma^t_j)
 * f^{gamma,t}_i = sum_j w_j (f^{gamma rho}_ij rho^t_j + 2 f^{gamma gamma}_ij gamma^t_j)
 * with gamma^t_j = grad rho_j . grad rho^t_j                           (Eq. frhot)
 * The four pair coefficients are written exactly as printed in Sec. II.B; their
 * delta_ij / w_i parts are added once per row (the j-sum weight w_i cancels 1/w_i).
 * rho_t: P x n, grad_rho_t: P x n x 3 (original indexing).
 * f_rho_t, f_gamma_t: P x n_rows. */
int orc_hessian_contract(int64_t n, const double* xyz, const double* w, const double* rho,
                         const double* grad, double b, double C, double rho_cut, int32_t P,
                         const double* rho_t, const double* grad_rho_t, int64_t n_rows,
                         const int64_t* rows, double* f_rho_t, double* f_gamma_t) {
    orc_sys s;
    if (orc_sys_init(&s, n, xyz, w, rho, grad, b, C, rho_cut)) return -1;
    int64_t nk = s.nk;
    /* trial values at kept points, j-major: rt[j*P + t], gt[j*P + t] */
    double* rt = (double*)malloc(sizeof(double) * (size_t)(nk > 0 ? nk : 1) * (P > 0 ? P : 1));
    double* gt = (double*)malloc(sizeof(double) * (size_t)(nk > 0 ? nk : 1) * (P > 0 ? P : 1));
    if (!rt || !gt) { free(rt); free(gt); orc_sys_free(&s); return -1; }
    for (int64_t j = 0; j < nk; ++j) {
        int64_t oj = s.kept[j];
        for (int32_t t = 0; t < P; ++t) {
            const double* gr = grad_rho_t + ((size_t)t * n + oj) * 3;
            rt[j * P + t] = rho_t[(size_t)t * n + oj];
            gt[j * P + t] = s.grad[3 * j] * gr[0] + s.grad[3 * j + 1] * gr[1] +
                            s.grad[3 * j + 2] * gr[2];
        }
    }
    int rc = 0;
#pragma omp parallel
    {
        nsum* acc = (nsum*)malloc(sizeof(nsum) * 2 * (size_t)(P > 0 ? P : 1));
        if (!acc) {
#pragma omp atomic write
            rc = -1;
        }
#pragma omp for schedule(dynamic, 2)
        for (int64_t r = 0; r < n_rows; ++r) {
            if (!acc) continue;
            int64_t oi = rows ? rows[r] : r;
            int64_t i = s.slot[oi];
            if (i < 0) {
                for (int32_t t = 0; t < P; ++t) {
                    f_rho_t[(size_t)t * n_rows + r] = 0.0;
                    f_gamma_t[(size_t)t * n_rows + r] = 0.0;
                }
                continue;
            }
            memset(acc, 0, sizeof(nsum) * 2 * (size_t)P);
            const orc_point* pi = &s.pt[i];
            for (int64_t j = 0; j < nk; ++j) {
                const orc_point* pj = &s.pt[j];
                double R2 = orc_r2(&s, i, j);
                double g = pi->omega * R2 + pi->kappa;
                double gp = pj->omega * R2 + pj->kappa;
                double sg = g + gp;
                double phi = -3.0 / (2.0 * g * gp * sg);
                double ai = R2 * pi->om_r + pi->ka_r;     /* d g  / d rho_i */
                double aj = R2 * pj->om_r + pj->ka_r;     /* d g' / d rho_j */
                double M = 2.0 / (sg * sg) + 2.0 / (g * gp);
                double f_rr = phi * (pi->rho * ai * pj->rho * aj * M
                                     - pi->rho * ai * (1.0 / sg + 1.0 / g)
                                     - pj->rho * aj * (1.0 / sg + 1.0 / gp) + 1.0);
                double f_gr = pi->rho * pi->om_g * R2 * phi *
                              (pj->rho * aj * M - (1.0 / sg + 1.0 / g));
                double f_rg = pj->rho * pj->om_g * R2 * phi *
                              (pi->rho * ai * M - (1.0 / sg + 1.0 / gp));
                double f_gg = pi->rho * pj->rho * pi->om_g * pj->om_g * R2 * R2 * phi * M;
                double wj = s.w[j];
                const double* rtj = rt + j * P;
                const double* gtj = gt + j * P;
                for (int32_t t = 0; t < P; ++t) {
                    nsum_add(&acc[t], wj * (f_rr * rtj[t] + 2.0 * f_rg * gtj[t]));
                    nsum_add(&acc[P + t], wj * (f_gr * rtj[t] + 2.0 * f_gg * gtj[t]));
                }
            }
            /* delta_ij / w_i parts of f^{rho rho}, f^{rho gamma} (= f^{gamma rho}), f^{gamma gamma} */
            double sums[6];
            orc_row_sums(&s, i, sums);
            double U = sums[1], W = sums[2], A = sums[3], B = sums[4], Cc = sums[5];
            const orc_point* p = pi;
            double d_rr = 2.0 * p->om_r * W + 2.0 * p->ka_r * U +
                          p->rho * (p->om_rr * W + p->ka_rr * U + p->ka_r * p->ka_r * A +
                                    p->om_r * p->om_r * Cc + 2.0 * p->om_r * p->ka_r * B);
            double d_rg = p->om_g * W + p->rho * p->om_rg * W + p->rho * p->om_g * p->ka_r * B +
                          p->rho * p->om_g * p->om_r * Cc;
            double d_gg = p->rho * (p->om_gg * W + p->om_g * p->om_g * Cc);
            for (int32_t t = 0; t < P; ++t) {
                double rti = rt[i * P + t], gti = gt[i * P + t];
                nsum_add(&acc[t], d_rr * rti + 2.0 * d_rg * gti);
                nsum_add(&acc[P + t], d_rg * rti + 2.0 * d_gg * gti);
                f_rho_t[(size_t)t * n_rows + r] = nsum_get(&acc[t]);
                f_gamma_t[(size_t)t * n_rows + r] = nsum_get(&acc[P + t]);
            }
        }
        free(acc);
    }
    free(rt);
    free(gt);
    orc_sys_free(&s);
    return rc;
}

/* ---------------------------------------------------------------- coordinate terms */
/* D_ij = omega_i/g + omega_j/g' + (omega_i + omega_j)/(g + g'), the bracket of Eq. grad_gr. */
static inline double orc_bracket(const orc_point* pi, const orc_point* pj, double g, double gp) {
    return pi->omega / g + pj->omega / gp + (pi->omega + pj->omega) / (g + gp);
}

/* Gradient of E with respect to the position of each grid point (rho, grad rho and w
 * held fixed): Eq. grad_gr with the atom A replaced by the single point i,
 *   dE/dr_i = -2 sum_j w_i w_j rho_i rho_j Phi_ij D_ij (r_i - r_j).
 * out: n_rows x 3. */
int orc_point_grad(int64_t n, const double* xyz, const double* w, const double* rho,
                   const double* grad, double b, double C, double rho_cut, int64_t n_rows,
                   const int64_t* rows, double* out) {
    orc_sys s;
    if (orc_sys_init(&s, n, xyz, w, rho, grad, b, C, rho_cut)) return -1;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t r = 0; r < n_rows; ++r) {
        int64_t oi = rows ? rows[r] : r;
        int64_t i = s.slot[oi];
        if (i < 0) { out[3 * r] = out[3 * r + 1] = out[3 * r + 2] = 0.0; continue; }
        nsum acc[3] = {{0, 0}, {0, 0}, {0, 0}};
        const orc_point* pi = &s.pt[i];
        double ci = s.w[i] * pi->rho;
        for (int64_t j = 0; j < s.nk; ++j) {
            const orc_point* pj = &s.pt[j];
            double R2 = orc_r2(&s, i, j);
            double g = pi->omega * R2 + pi->kappa;
            double gp = pj->omega * R2 + pj->kappa;
            double phi = -3.0 / (2.0 * g * gp * (g + gp));
            double f = -2.0 * ci * s.w[j] * pj->rho * phi * orc_bracket(pi, pj, g, gp);
            for (int d = 0; d < 3; ++d) nsum_add(&acc[d], f * (s.xyz[3 * i + d] - s.xyz[3 * j + d]));
        }
        for (int d = 0; d < 3; ++d) out[3 * r + d] = nsum_get(&acc[d]);
    }
    orc_sys_free(&s);
    return 0;
}

/* E^A_gr for every atom, the first form of Eq. grad_gr: two double sums,
 * over (i in A, j not in A) and (i not in A, j in A).  out: n_atom x 3. */
int orc_atom_grad(int64_t n, const double* xyz, const double* w, const double* rho,
                  const double* grad, const int32_t* atom_of_point, int32_t n_atom, double b,
                  double C, double rho_cut, double* out) {
    orc_sys s;
    if (orc_sys_init(&s, n, xyz, w, rho, grad, b, C, rho_cut)) return -1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t A = 0; A < n_atom; ++A) {
        nsum acc[3] = {{0, 0}, {0, 0}, {0, 0}};
        for (int64_t i = 0; i < s.nk; ++i) {
            int inA = atom_of_point[s.kept[i]] == A;
            for (int64_t j = 0; j < s.nk; ++j) {
                int jnA = atom_of_point[s.kept[j]] == A;
                if (inA == jnA) continue;
                const orc_point* pi = &s.pt[i];
                const orc_point* pj = &s.pt[j];
                double R2 = orc_r2(&s, i, j);
                double g = pi->omega * R2 + pi->kappa;
                double gp = pj->omega * R2 + pj->kappa;
                double phi = -3.0 / (2.0 * g * gp * (g + gp));
                double f = -s.w[i] * s.w[j] * pi->rho * pj->rho * phi * orc_bracket(pi, pj, g, gp);
                for (int d = 0; d < 3; ++d) {
                    double dr = inA ? (s.xyz[3 * i + d] - s.xyz[3 * j + d])   /* first line  */
                                    : (s.xyz[3 * j + d] - s.xyz[3 * i + d]);  /* second line */
                    nsum_add(&acc[d], f * dr);
                }
            }
        }
        for (int d = 0; d < 3; ++d) out[3 * A + d] = nsum_get(&acc[d]);
    }
    orc_sys_free(&s);
    return 0;
}

/* E_i^{Bgr}, U_i^{Bgr}, W_i^{Bgr} (Eq. EiBgr and the two equations after it):
 * for i not in B a sum over j in B; for i in B minus the sum over the other atoms.
 * out_E, out_U, out_W: n_rows x n_atom x 3. */
int orc_atom_resolved(int64_t n, const double* xyz, const double* w, const double* rho,
                      const double* grad, const int32_t* atom_of_point, int32_t n_atom,
                      double b, double C, double rho_cut, int64_t n_rows, const int64_t* rows,
                      double* out_E, double* out_U, double* out_W) {
    orc_sys s;
    if (orc_sys_init(&s, n, xyz, w, rho, grad, b, C, rho_cut)) return -1;
    int rc = 0;
#pragma omp parallel
    {
        nsum* acc = (nsum*)malloc(sizeof(nsum) * 9 * (size_t)n_atom);
        if (!acc) {
#pragma omp atomic write
            rc = -1;
        }
#pragma omp for schedule(dynamic, 4)
        for (int64_t r = 0; r < n_rows; ++r) {
            if (!acc) continue;
            int64_t oi = rows ? rows[r] : r;
            int64_t i = s.slot[oi];
            double* oE = out_E + (size_t)r * n_atom * 3;
            double* oU = out_U + (size_t)r * n_atom * 3;
            double* oW = out_W + (size_t)r * n_atom * 3;
            if (i < 0) {
                memset(oE, 0, sizeof(double) * 3 * n_atom);
                memset(oU, 0, sizeof(double) * 3 * n_atom);
                memset(oW, 0, sizeof(double) * 3 * n_atom);
                continue;
            }
            memset(acc, 0, sizeof(nsum) * 9 * (size_t)n_atom);
            int Ai = atom_of_point[oi];
            const orc_point* pi = &s.pt[i];
            for (int64_t j = 0; j < s.nk; ++j) {
                int Bj = atom_of_point[s.kept[j]];
                if (Bj == Ai) continue;   /* the i in B case is filled below */
                const orc_point* pj = &s.pt[j];
                double R2 = orc_r2(&s, i, j);
                double g = pi->omega * R2 + pi->kappa;
                double gp = pj->omega * R2 + pj->kappa;
                double sg = g + gp;
                double phi = -3.0 / (2.0 * g * gp * sg);
                double cj = s.w[j] * pj->rho;
                double D = orc_bracket(pi, pj, g, gp);
                double t1 = 1.0 / sg + 1.0 / g;
                double t3 = pi->omega / (g * g) + (pi->omega + pj->omega) / (sg * sg);
                double fE = -2.0 * cj * phi * D;
                double fU = 2.0 * cj * phi * (D * t1 + t3);
                double fW = 2.0 * cj * phi * (R2 * D * t1 + R2 * t3 - t1);
                for (int d = 0; d < 3; ++d) {
                    double dr = s.xyz[3 * j + d] - s.xyz[3 * i + d];
                    nsum_add(&acc[9 * Bj + d], fE * dr);
                    nsum_add(&acc[9 * Bj + 3 + d], fU * dr);
                    nsum_add(&acc[9 * Bj + 6 + d], fW * dr);
                }
            }
            for (int32_t B = 0; B < n_atom; ++B)
                for (int d = 0; d < 3; ++d) {
                    oE[3 * B + d] = nsum_get(&acc[9 * B + d]);
                    oU[3 * B + d] = nsum_get(&acc[9 * B + 3 + d]);
                    oW[3 * B + d] = nsum_get(&acc[9 * B + 6 + d]);
                }
            if (Ai >= 0 && Ai < n_atom) {
                nsum e[3] = {{0, 0}, {0, 0}, {0, 0}}, u[3] = {{0, 0}, {0, 0}, {0, 0}},
                     v[3] = {{0, 0}, {0, 0}, {0, 0}};
                for (int32_t B = 0; B < n_atom; ++B) {
                    if (B == Ai) continue;
                    for (int d = 0; d < 3; ++d) {
                        nsum_add(&e[d], -oE[3 * B + d]);
                        nsum_add(&u[d], -oU[3 * B + d]);
                        nsum_add(&v[d], -oW[3 * B + d]);
                    }
                }
                for (int d = 0; d < 3; ++d) {
                    oE[3 * Ai + d] = nsum_get(&e[d]);
                    oU[3 * Ai + d] = nsum_get(&u[d]);
                    oW[3 * Ai + d] = nsum_get(&v[d]);
                }
            }
        }
        free(acc);
    }
    orc_sys_free(&s);
    return rc;
}

/* D_i^B, the three-by-three matrix of the grid-grid block (Sec. II.B, the equation for
 * D_i^B), for i not in B:
 *   D_i^B = -2 sum_{j in B} w_j rho_j Phi_ij [ 2 (D^2 + (omega_i/g)^2 + (omega_j/g')^2
 *           + ((omega_i+omega_j)/(g+g'))^2) (r_j - r_i)(r_j - r_i)^T - D I_3 ],
 * D the bracket of Eq. grad_gr.  pair_D adds the j term into acc[9] (row-major 3x3). */
static void orc_pair_D(const orc_sys* s, int64_t i, int64_t j, nsum acc[9]) {
    const orc_point* pi = &s->pt[i];
    const orc_point* pj = &s->pt[j];
    double R2 = orc_r2(s, i, j);
    double g = pi->omega * R2 + pi->kappa;
    double gp = pj->omega * R2 + pj->kappa;
    double sg = g + gp;
    double phi = -3.0 / (2.0 * g * gp * sg);
    double D = orc_bracket(pi, pj, g, gp);
    double a = pi->omega / g, bb = pj->omega / gp, c = (pi->omega + pj->omega) / sg;
    double sq = 2.0 * (D * D + a * a + bb * bb + c * c);
    double pre = -2.0 * s->w[j] * pj->rho * phi;
    double dr[3];
    for (int d = 0; d < 3; ++d) dr[d] = s->xyz[3 * j + d] - s->xyz[3 * i + d];
    for (int u = 0; u < 3; ++u)
        for (int v = 0; v < 3; ++v)
            nsum_add(&acc[3 * u + v], pre * (sq * dr[u] * dr[v] - (u == v ? D : 0.0)));
}

/* D_i^B for selected rows: out n_rows x n_atom x 9 (zero for B = atom(i) and for rows
 * below the cutoff). */
int orc_point_coord_hessian(int64_t n, const double* xyz, const double* w, const double* rho,
                            const double* grad, const int32_t* atom_of_point, int32_t n_atom,
                            double b, double C, double rho_cut, int64_t n_rows,
                            const int64_t* rows, double* out) {
    orc_sys s;
    if (orc_sys_init(&s, n, xyz, w, rho, grad, b, C, rho_cut)) return -1;
    int rc = 0;
#pragma omp parallel
    {
        nsum* acc = (nsum*)malloc(sizeof(nsum) * 9 * (size_t)n_atom);
        if (!acc) {
#pragma omp atomic write
            rc = -1;
        }
#pragma omp for schedule(dynamic, 4)
        for (int64_t r = 0; r < n_rows; ++r) {
            if (!acc) continue;
            int64_t oi = rows ? rows[r] : r;
            int64_t i = s.slot[oi];
            double* o = out + (size_t)r * n_atom * 9;
            memset(o, 0, sizeof(double) * 9 * (size_t)n_atom);
            if (i < 0) continue;
            memset(acc, 0, sizeof(nsum) * 9 * (size_t)n_atom);
            int Ai = atom_of_point[oi];
            for (int64_t j = 0; j < s.nk; ++j) {
                int Bj = atom_of_point[s.kept[j]];
                if (Bj == Ai) continue;
                orc_pair_D(&s, i, j, &acc[9 * Bj]);
            }
            for (int32_t B = 0; B < n_atom; ++B)
                if (B != Ai)
                    for (int q = 0; q < 9; ++q) o[9 * B + q] = nsum_get(&acc[9 * B + q]);
        }
        free(acc);
    }
    orc_sys_free(&s);
    return rc;
}

/* E^{AB}_{gr,gr} = sum_{i in A} w_i rho_i D_i^B for A != B, and E^{AA}_{gr,gr} = minus the
 * sum over B != A (Sec. II.B): out n_atom x n_atom x 9, block (A, B) row-major 3x3. */
int orc_coord_hessian(int64_t n, const double* xyz, const double* w, const double* rho,
                      const double* grad, const int32_t* atom_of_point, int32_t n_atom, double b,
                      double C, double rho_cut, double* out) {
    orc_sys s;
    if (orc_sys_init(&s, n, xyz, w, rho, grad, b, C, rho_cut)) return -1;
    int rc = 0;
#pragma omp parallel
    {
        nsum* acc = (nsum*)malloc(sizeof(nsum) * 9 * (size_t)n_atom);
        nsum* dB = (nsum*)malloc(sizeof(nsum) * 9 * (size_t)n_atom);
        if (!acc || !dB) {
#pragma omp atomic write
            rc = -1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int32_t A = 0; A < n_atom; ++A) {
            if (!acc || !dB) continue;
            memset(acc, 0, sizeof(nsum) * 9 * (size_t)n_atom);
            for (int64_t i = 0; i < s.nk; ++i) {
                if (atom_of_point[s.kept[i]] != A) continue;
                memset(dB, 0, sizeof(nsum) * 9 * (size_t)n_atom);
                for (int64_t j = 0; j < s.nk; ++j) {
                    int Bj = atom_of_point[s.kept[j]];
                    if (Bj == A) continue;
                    orc_pair_D(&s, i, j, &dB[9 * Bj]);
                }
                double ci = s.w[i] * s.pt[i].rho;
                for (int32_t B = 0; B < n_atom; ++B)
                    for (int q = 0; q < 9; ++q) nsum_add(&acc[9 * B + q], ci * nsum_get(&dB[9 * B + q]));
            }
            double* o = out + (size_t)A * n_atom * 9;
            for (int32_t B = 0; B < n_atom; ++B)
                for (int q = 0; q < 9; ++q) o[9 * B + q] = (B == A) ? 0.0 : nsum_get(&acc[9 * B + q]);
            for (int q = 0; q < 9; ++q) {
                nsum d = {0, 0};
                for (int32_t B = 0; B < n_atom; ++B)
                    if (B != A) nsum_add(&d, -o[9 * B + q]);
                o[9 * A + q] = nsum_get(&d);
            }
        }
        free(acc);
        free(dB);
    }
    orc_sys_free(&s);
    return rc;
}

/* ---------------------------------------------------------------- weight-derivative sums */
/* E_i^{Bw}, U_i^{Bw}, W_i^{Bw} (Sec. II.B, the three sums printed after the nuclear-Hessian
 * blocks) for P weight directions: with v_j = wt[p][j] in place of w_j^B,
 *   E_i^v = sum_j v_j rho_j Phi_ij
 *   U_i^v = -sum_j v_j rho_j Phi_ij (1/(g + g') + 1/g)
 *   W_i^v = -sum_j v_j rho_j Phi_ij R^2 (1/(g + g') + 1/g),
 * the sums E_i, U_i, W_i of Sec. II.A with v in place of w (j = i included, kept points
 * only).  wt: P x n (caller order); outE/outU/outW: P x n_rows, zero for dropped rows. */
int orc_weight_response(int64_t n, const double* xyz, const double* w, const double* rho,
                        const double* grad, double b, double C, double rho_cut, int32_t P,
                        const double* wt, int64_t n_rows, const int64_t* rows, double* outE,
                        double* outU, double* outW) {
    orc_sys s;
    if (orc_sys_init(&s, n, xyz, w, rho, grad, b, C, rho_cut)) return -1;
    int rc = 0;
#pragma omp parallel
    {
        nsum* acc = (nsum*)malloc(sizeof(nsum) * 3 * (size_t)(P > 0 ? P : 1));
        if (!acc) {
#pragma omp atomic write
            rc = -1;
        }
#pragma omp for schedule(dynamic, 4)
        for (int64_t r = 0; r < n_rows; ++r) {
            if (!acc) continue;
            int64_t oi = rows ? rows[r] : r;
            int64_t i = s.slot[oi];
            memset(acc, 0, sizeof(nsum) * 3 * (size_t)P);
            if (i >= 0) {
                const orc_point* pi = &s.pt[i];
                for (int64_t j = 0; j < s.nk; ++j) {
                    const orc_point* pj = &s.pt[j];
                    double R2 = orc_r2(&s, i, j);
                    double g = pi->omega * R2 + pi->kappa;
                    double gp = pj->omega * R2 + pj->kappa;
                    double sg = g + gp;
                    double phi = -3.0 / (2.0 * g * gp * sg);
                    double t1 = 1.0 / sg + 1.0 / g;
                    int64_t oj = s.kept[j];
                    for (int32_t p = 0; p < P; ++p) {
                        double vj = wt[(size_t)p * n + oj] * pj->rho;
                        nsum_add(&acc[3 * p], vj * phi);
                        nsum_add(&acc[3 * p + 1], -vj * phi * t1);
                        nsum_add(&acc[3 * p + 2], -vj * phi * R2 * t1);
                    }
                }
            }
            for (int32_t p = 0; p < P; ++p) {
                outE[(size_t)p * n_rows + r] = nsum_get(&acc[3 * p]);
                outU[(size_t)p * n_rows + r] = nsum_get(&acc[3 * p + 1]);
                outW[(size_t)p * n_rows + r] = nsum_get(&acc[3 * p + 2]);
            }
        }
        free(acc);
    }
    orc_sys_free(&s);
    return rc;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int k) {
#ifdef _OPENMP
    if (k > 0) omp_set_num_threads(k);
#else
    (void)k;
#endif
}
