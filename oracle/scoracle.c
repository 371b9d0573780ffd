/*
 * scoracle.c -- plain, slow, FP64 CPU oracle for the semi-coherent search
 * statistic of Bandopadhyay & Moore, arXiv:2408.13170.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file:
 * it is imported by tests/, by __graft_entry__.smoke() and by the
 * cpu_baseline / reference leg of bench.py, and by nothing else.
 *
 * It shares no code with the CUDA library.  Every quantity is evaluated per
 * frequency bin straight from its definition:
 *
 *   inner product   <a|b> = sum_alpha 4 Re int a_alpha conj(b_alpha)/S_alpha df
 *                                                  (Sec. II.A, Eq. inner_prod)
 *   segment product [a|b]_n = same sum restricted to [f_n, f_{n+1})
 *                                                  (Sec. II.B)
 *   x_n = max_phi [d|h e^{i phi}]_n = |z_n|,  z_n = sum 4 df d conj(h)/S
 *                                                  (Sec. II.B, Eq. semi-coherent_O)
 *   Upsilon_N = sum_n x_n^2 / [h|h]_n             (Sec. II.B, Upsilon_N)
 *   equal squared-SNR segment boundaries          (Sec. II.B, last paragraph)
 *   waveform: (2,2)-mode frequency-domain PN inspiral, h = A e^{-i Psi}
 *                                                  (Sec. IV, TaylorF2 family)
 *   response: h_alpha = T_alpha(theta, f) h        (Sec. IV, LISA TDI A, E
 *                                                  and, optionally, T: the
 *                                                  search uses all three
 *                                                  channels, Sec. I)
 *
 * Readings where the paper is silent:
 *   - waveform: the paper's TaylorF2Ecc (Sec. IV) is not printed.  Read as
 *     the non-spinning TaylorF2 phase to 3.5PN (orders v^0..v^7 of the
 *     energy-balance SPA phase, with the 2.5PN term written
 *     phi_5 (1 + 3 ln(v/v_lso)), v_lso = 6^{-1/2}, and the 3PN logarithm
 *     ln(4v)) plus the leading-order eccentric correction
 *     -(2355/1462) e0^2 chi^{-19/9} times the Newtonian term, chi = f/f0,
 *     e0 the eccentricity at the particle's initial frequency f0 (Yunes,
 *     Arun, Berti & Will 2009: the O(e0^2) SPA phase of the Peters-Mathews
 *     inspiral); 0 <= e0 <= 0.3; t(f) is defined as Psi'(f)/(2 pi); t_c
 *     fixed by t(f0) = 0; hard support cut f >= f0, t(f) <= T_obs,
 *     v <= 6^{-1/2};
 *   - response: rigid-adiabatic single-link transfer from the two-pulse
 *     link formula, evaluated at t = t(f), first-generation TDI X,Y,Z and
 *     A = (Z-X)/sqrt2, E = (X-2Y+Z)/sqrt6, T = (X+Y+Z)/sqrt3 (the
 *     orthonormal combinations), on an exactly rigid equal-arm
 *     orbit with the constellation centre at (R cos Omega t, R sin Omega t, 0);
 *   - equal-SNR^2 segments: trapezoid cumulative of the exact template
 *     power on an anchor grid of stride 1024 bins, linear inverse
 *     interpolation, bin k in segment n iff kappa_n <= k < kappa_{n+1},
 *     with each interior kappa_n lowered by 2^-20 bins: a kappa that is an
 *     integer in exact arithmetic (a support shorter than one anchor stride
 *     makes kappa_n = k_lo + n (k_hi - k_lo)/N) then starts its segment at
 *     that integer whatever the last bit of its FP64 rounding;
 *   - the large waveform phase (up to ~1e8 rad) is evaluated in
 *     double-double arithmetic, reduced modulo one turn, then rounded.
 *
 * Sums over bins are Neumaier-compensated.  OpenMP parallelises over
 * particles only; the arithmetic per particle is sequential.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -fPIC -shared (no FMA contraction:
 * the double-double routines rely on separately rounded products).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* physical constants (seconds)                                        */
/* ------------------------------------------------------------------ */
#define ORC_TSUN 4.925490947641267e-6            /* G Msun / c^3 [s] */
#define ORC_CLIGHT 299792458.0
#define ORC_ARM (2.5e9 / ORC_CLIGHT)             /* L [s] */
#define ORC_AU (149597870700.0 / ORC_CLIGHT)      /* R [s] */
#define ORC_YEAR 3.15581497632e7                  /* sidereal year [s] */

enum { ORC_TF2 = 0, ORC_NEWTONIAN = 1, ORC_LINEAR_CHIRP = 2 };
enum { ORC_TDI_AE = 0, ORC_IDENTITY = 1 };
enum { ORC_EQUAL_WIDTH = 0, ORC_EQUAL_SNR2 = 1 };
enum { ORC_OK = 0, ORC_INVALID = 1, ORC_EMPTY = 2 };

/* ------------------------------------------------------------------ */
/* double-double arithmetic (error-free transformations)               */
/* ------------------------------------------------------------------ */
typedef struct { double hi, lo; } dd;

static dd mk(double hi, double lo) { dd r; r.hi = hi; r.lo = lo; return r; }
static dd from_d(double a) { return mk(a, 0.0); }

static dd two_sum(double a, double b) {
    double s = a + b;
    double bv = s - a;
    double av = s - bv;
    return mk(s, (a - av) + (b - bv));
}
static dd fast_two_sum(double a, double b) {   /* |a| >= |b| */
    double s = a + b;
    return mk(s, b - (s - a));
}
static dd two_prod(double a, double b) {
    double p = a * b;
    return mk(p, fma(a, b, -p));
}
static dd dd_add(dd a, dd b) {
    dd s = two_sum(a.hi, b.hi);
    dd t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}
static dd dd_neg(dd a) { return mk(-a.hi, -a.lo); }
static dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
static dd dd_mul(dd a, dd b) {
    dd p = two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo + a.lo * b.hi;
    return fast_two_sum(p.hi, p.lo);
}
static dd dd_mul_d(dd a, double b) { return dd_mul(a, from_d(b)); }
static dd dd_div(dd a, dd b) {
    double q1 = a.hi / b.hi;
    dd r = dd_sub(a, dd_mul_d(b, q1));
    double q2 = r.hi / b.hi;
    r = dd_sub(r, dd_mul_d(b, q2));
    double q3 = r.hi / b.hi;
    dd q = fast_two_sum(q1, q2);
    return dd_add(q, from_d(q3));
}
static double dd_to_d(dd a) { return a.hi + a.lo; }

/* pi as a double-double */
static const dd DD_PI = {3.141592653589793116e+00, 1.224646799147353207e-16};

/* y = x^(-1/3) for x > 0: double estimate, two Newton steps in double-double
 * on g(y) = y^3 x - 1. */
static dd dd_rcbrt(dd x) {
    dd y = from_d(1.0 / cbrt(x.hi));
    for (int it = 0; it < 2; ++it) {
        dd y3x = dd_mul(dd_mul(dd_mul(y, y), y), x);
        dd r = dd_sub(from_d(1.0), y3x);            /* 1 - y^3 x */
        y = dd_add(y, dd_mul(y, dd_div(r, from_d(3.0))));
    }
    return y;
}
/* y = x^(-3/5) for x > 0: Newton on g(y) = y^5 x^3 - 1 */
static dd dd_pow_m35(dd x) {
    dd y = from_d(pow(x.hi, -0.6));
    dd x3 = dd_mul(dd_mul(x, x), x);
    for (int it = 0; it < 2; ++it) {
        dd y2 = dd_mul(y, y);
        dd y5 = dd_mul(dd_mul(y2, y2), y);
        dd r = dd_sub(from_d(1.0), dd_mul(y5, x3));
        y = dd_add(y, dd_mul(y, dd_div(r, from_d(5.0))));
    }
    return y;
}

/* ------------------------------------------------------------------ */
/* particle: the source parameters and everything derived from them    */
/* ------------------------------------------------------------------ */
typedef struct {
    int waveform, response;
    /* raw parameters theta = {Mc, q, f0, lambda, beta, iota, psi, e0} */
    double th[8];
    /* PN waveform */
    dd eta, Ms;            /* symmetric mass ratio; total mass in seconds */
    dd phi2, phi3, phi4;   /* PN phase coefficients (phi0 = 1) */
    double phi5;           /* 2.5PN: phi5 (1 + 3 ln(v/v_lso)) */
    double phi6c, phi6l;   /* 3PN: phi6c + phi6l ln(4v) */
    double phi7;           /* 3.5PN */
    dd ecc;                /* -(2355/1462) e0^2 f0^{19/9} (0 when circular) */
    dd piMs;               /* pi * Ms */
    dd tc;                 /* coalescence time, fixed by t(f0) = 0 */
    double fdot;           /* linear-chirp test model: df/dt */
    /* response */
    double kvec[3];                /* propagation direction */
    double complex P[3][3];        /* complex polarisation tensor */
} orc_particle;

/* The PN phase split by order.  With P = 3/(256 pi eta) and v = (pi M f)^{1/3}
 * (Sec. IV, TaylorF2 family), in turns:
 *   F_k = P phi_k v^{k-5}                      k = 0, 2, 3, 4, 7
 *   F_5 = P phi5 (1 + 3 ln(v/v_lso))
 *   F_6 = P v (phi6c + phi6l ln(4v))
 *   F_e = P ecc v^{-5} f^{-19/9}  (= Newtonian x -(2355/1462) e0^2 (f/f0)^{-19/9})
 * and the time terms t_j = dF_j/df (d v/df = v/(3f)):
 *   t_k = F_k (k-5)/(3f),   t_5 = P phi5/f,
 *   t_6 = P v (phi6c + phi6l ln(4v) + phi6l)/(3f),   t_e = -(34/9) F_e/f.
 * F[j], T[j] for j = 0..7 <-> orders 0, 1, 1.5, 2, 2.5, 3, 3.5PN and the
 * eccentric term.  The Newtonian model keeps j = 0 only (its other
 * coefficients are zero).  The large terms (j = 0..3, e) are double-double;
 * the 2.5-3.5PN terms (|F| below ~1e3 turns) are plain doubles. */
static void pn_terms(const orc_particle *p, dd f, dd F[8], dd T[8]) {
    dd y = dd_rcbrt(dd_mul(p->piMs, f));               /* 1/v */
    dd P = dd_div(from_d(3.0), dd_mul(dd_mul_d(DD_PI, 256.0), p->eta));
    dd y2 = dd_mul(y, y);
    dd y3 = dd_mul(y2, y);
    dd y5 = dd_mul(y3, y2);
    dd inv3f = dd_div(from_d(1.0), dd_mul_d(f, 3.0));  /* 1/(3f) */
    const dd pw[4] = {y5, y3, y2, y};                   /* v^{k-5}, k=0,2,3,4 */
    const dd phk[4] = {from_d(1.0), p->phi2, p->phi3, p->phi4};
    const double km5[4] = {-5.0, -3.0, -2.0, -1.0};
    for (int j = 0; j < 4; ++j) {
        F[j] = dd_mul(dd_mul(P, phk[j]), pw[j]);
        T[j] = dd_mul_d(dd_mul(F[j], inv3f), km5[j]);
    }
    double v = 1.0 / dd_to_d(y), Pd = dd_to_d(P), fd = dd_to_d(f);
    double lnv = log(v);
    /* 2.5PN */
    double F5 = Pd * p->phi5 * (1.0 + 3.0 * (lnv + 0.5 * log(6.0)));
    F[4] = from_d(F5);
    T[4] = from_d(Pd * p->phi5 / fd);
    /* 3PN */
    double br6 = p->phi6c + p->phi6l * (log(4.0) + lnv);
    F[5] = from_d(Pd * v * br6);
    T[5] = from_d(Pd * v * (br6 + p->phi6l) / (3.0 * fd));
    /* 3.5PN */
    double F7 = Pd * p->phi7 * v * v;
    F[6] = from_d(F7);
    T[6] = from_d(F7 * 2.0 / (3.0 * fd));
    /* eccentric: f^{-19/9} = f^{-2} f^{-1/9}, f^{-1/9} = (f^{1/3})^{-1/3} */
    if (p->ecc.hi != 0.0) {
        dd f13 = dd_div(from_d(1.0), dd_rcbrt(f));
        dd fm19 = dd_mul(dd_rcbrt(f13), dd_div(from_d(1.0), dd_mul(f, f)));
        F[7] = dd_mul(dd_mul(dd_mul(P, p->ecc), y5), fm19);
        T[7] = dd_div(dd_mul_d(F[7], -34.0), dd_mul_d(f, 9.0));
    } else {
        F[7] = from_d(0.0);
        T[7] = from_d(0.0);
    }
}

/* t(f) - t_c = sum of the time terms                         [seconds, dd] */
static dd pn_time_offset(const orc_particle *p, dd f) {
    dd F[8], T[8];
    pn_terms(p, f, F, T);
    dd s = T[0];
    for (int j = 1; j < 8; ++j) s = dd_add(s, T[j]);
    return s;
}

/* Psi(f)/(2 pi) in turns, before adding f t_c and -1/8        [turns, dd] */
static dd pn_phase_turns(const orc_particle *p, dd f) {
    dd F[8], T[8];
    pn_terms(p, f, F, T);
    dd s = F[0];
    for (int j = 1; j < 8; ++j) s = dd_add(s, F[j]);
    return s;
}

static int finite8(const double *th) {
    for (int i = 0; i < 8; ++i)
        if (!isfinite(th[i])) return 0;
    return 1;
}

/* Derive the particle; returns ORC_OK or ORC_INVALID. */
static int particle_init(orc_particle *p, const double *th, int waveform,
                         int response) {
    memset(p, 0, sizeof(*p));
    p->waveform = waveform;
    p->response = response;
    memcpy(p->th, th, sizeof(p->th));
    if (!finite8(th)) return ORC_INVALID;
    double Mc = th[0], q = th[1], f0 = th[2];
    double e0 = th[7];
    if (f0 <= 0.0) return ORC_INVALID;
    /* eccentricity: TaylorF2 only, 0 <= e0 <= 0.3 */
    if (e0 != 0.0 && (waveform != ORC_TF2 || !(e0 > 0.0 && e0 <= 0.3)))
        return ORC_INVALID;
    if (waveform == ORC_LINEAR_CHIRP) {
        if (Mc <= 0.0) return ORC_INVALID;
        p->fdot = Mc;
    } else {
        if (Mc <= 0.0 || q < 1.0) return ORC_INVALID;
        /* eta = q/(1+q)^2, M = Mc eta^{-3/5} */
        dd onepq = two_sum(1.0, q);
        p->eta = dd_div(from_d(q), dd_mul(onepq, onepq));
        p->Ms = dd_mul_d(dd_mul(from_d(Mc), dd_pow_m35(p->eta)), ORC_TSUN);
        p->piMs = dd_mul(DD_PI, p->Ms);
        if (waveform == ORC_TF2) {
            dd e = p->eta;
            p->phi2 = dd_add(dd_div(from_d(3715.0), from_d(756.0)),
                             dd_mul(dd_div(from_d(55.0), from_d(9.0)), e));
            p->phi3 = dd_mul_d(DD_PI, -16.0);
            p->phi4 = dd_add(
                dd_add(dd_div(from_d(15293365.0), from_d(508032.0)),
                       dd_mul(dd_div(from_d(27145.0), from_d(504.0)), e)),
                dd_mul(dd_div(from_d(3085.0), from_d(72.0)), dd_mul(e, e)));
            double et = dd_to_d(e), pi = M_PI, gE = 0.57721566490153286061;
            p->phi5 = pi * (38645.0 / 756.0 - 65.0 / 9.0 * et);
            p->phi6c = 11583231236531.0 / 4694215680.0 - 640.0 / 3.0 * pi * pi
                       - 6848.0 / 21.0 * gE
                       + (-15737765635.0 / 3048192.0 + 2255.0 / 12.0 * pi * pi) * et
                       + 76055.0 / 1728.0 * et * et
                       - 127825.0 / 1296.0 * et * et * et;
            p->phi6l = -6848.0 / 21.0;
            p->phi7 = pi * (77096675.0 / 254016.0 + 378515.0 / 1512.0 * et
                            - 74045.0 / 756.0 * et * et);
            /* -(2355/1462) e0^2 f0^{19/9}; f0^{19/9} = f0^2 (f0^{1/3})^{1/3} */
            if (e0 != 0.0) {
                dd f0d = from_d(f0);
                dd f013 = dd_div(from_d(1.0), dd_rcbrt(f0d));
                dd f019 = dd_div(from_d(1.0), dd_rcbrt(f013));
                dd c = dd_div(from_d(-2355.0), from_d(1462.0));
                p->ecc = dd_mul(dd_mul(c, dd_mul(from_d(e0), from_d(e0))),
                                dd_mul(dd_mul(f0d, f0d), f019));
            }
        } else {
            p->phi2 = from_d(0.0);
            p->phi3 = from_d(0.0);
            p->phi4 = from_d(0.0);
        }
        /* beyond the last stable orbit already at f0 -> non-physical */
        if (dd_to_d(p->piMs) * f0 > pow(6.0, -1.5)) return ORC_INVALID;
        /* t(f0) = 0  =>  t_c = -(t(f0) - t_c) */
        p->tc = dd_neg(pn_time_offset(p, from_d(f0)));
    }
    /* sky and polarisation */
    double lam = th[3], bet = th[4], inc = th[5], psi = th[6];
    double k[3] = {-cos(bet) * cos(lam), -cos(bet) * sin(lam), -sin(bet)};
    double u[3] = {sin(lam), -cos(lam), 0.0};
    double v[3] = {-sin(bet) * cos(lam), -sin(bet) * sin(lam), cos(bet)};
    memcpy(p->kvec, k, sizeof(k));
    double c2p = cos(2.0 * psi), s2p = sin(2.0 * psi);
    double ap = 0.5 * (1.0 + cos(inc) * cos(inc));
    double ax = cos(inc);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double ep = u[i] * u[j] - v[i] * v[j];
            double ex = u[i] * v[j] + v[i] * u[j];
            double Ep = c2p * ep + s2p * ex;
            double Ex = -s2p * ep + c2p * ex;
            p->P[i][j] = ap * Ep - I * ax * Ex;
        }
    return ORC_OK;
}

/* f_k = f_first + k df, exactly, as a double-double */
static dd grid_freq(double f_first, double df, int64_t k) {
    return dd_add(from_d(f_first), two_prod((double)k, df));
}

/* time-to-frequency map t(f) (double) */
static double time_of_freq(const orc_particle *p, dd f) {
    if (p->waveform == ORC_LINEAR_CHIRP)
        return (dd_to_d(f) - p->th[2]) / p->fdot;
    return dd_to_d(dd_add(p->tc, pn_time_offset(p, f)));
}

/* waveform phase Psi(f)/(2 pi) reduced to [-1/2, 1/2] turns */
static double phase_turns_reduced(const orc_particle *p, dd f) {
    dd F;
    if (p->waveform == ORC_LINEAR_CHIRP) {
        /* (f - f0)^2 / (2 fdot) - 1/8 */
        dd x = dd_sub(f, from_d(p->th[2]));
        F = dd_div(dd_mul(x, x), from_d(2.0 * p->fdot));
    } else {
        F = dd_add(dd_mul(f, p->tc), pn_phase_turns(p, f));
    }
    F = dd_sub(F, from_d(0.125));
    double n = nearbyint(F.hi);
    return dd_to_d(dd_sub(F, from_d(n)));
}

/* support test of one bin (the bin already satisfies f_k >= f0) */
static int in_band(const orc_particle *p, dd f, double T_obs) {
    if (p->waveform != ORC_LINEAR_CHIRP) {
        if (dd_to_d(p->piMs) * dd_to_d(f) > pow(6.0, -1.5)) return 0;
    }
    return time_of_freq(p, f) <= T_obs;
}

/* ------------------------------------------------------------------ */
/* LISA: rigid equal-arm orbit and the TDI response                    */
/* ------------------------------------------------------------------ */
static void orbit(double t, double pos[3][3]) {
    const double R = ORC_AU;
    const double e = ORC_ARM / (2.0 * sqrt(3.0) * R);
    double a = 2.0 * M_PI / ORC_YEAR * t;
    for (int i = 0; i < 3; ++i) {
        double b = 2.0 * M_PI * i / 3.0;
        pos[i][0] = R * cos(a) + 0.5 * e * R * (cos(2.0 * a - b) - 3.0 * cos(b));
        pos[i][1] = R * sin(a) + 0.5 * e * R * (sin(2.0 * a - b) - 3.0 * sin(b));
        pos[i][2] = -sqrt(3.0) * e * R * cos(a - b);
    }
}

/* single-link transfer s -> r (0-based craft indices) */
static double complex link(const orc_particle *p, double pos[3][3], int s,
                           int r, double f) {
    const double L = ORC_ARM;
    double n[3], kn = 0.0, kp = 0.0;
    for (int i = 0; i < 3; ++i) {
        n[i] = (pos[r][i] - pos[s][i]) / L;
        kn += p->kvec[i] * n[i];
        kp += p->kvec[i] * (pos[s][i] + pos[r][i]);
    }
    double complex nPn = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) nPn += n[i] * p->P[i][j] * n[j];
    double x = M_PI * f * L * (1.0 - kn);
    double sinc = (x == 0.0) ? 1.0 : sin(x) / x;
    double ph = -M_PI * f * (L + kp);
    return -I * M_PI * f * L * sinc * cexp(I * ph) * nPn;
}

/* out: G[6] (links 1->2,2->1,1->3,3->1,2->3,3->2), X, Y, Z, A, E, T */
static void tdi(const orc_particle *p, double f, double t,
                double complex out[12]) {
    double pos[3][3];
    orbit(t, pos);
    double complex G12 = link(p, pos, 0, 1, f), G21 = link(p, pos, 1, 0, f);
    double complex G13 = link(p, pos, 0, 2, f), G31 = link(p, pos, 2, 0, f);
    double complex G23 = link(p, pos, 1, 2, f), G32 = link(p, pos, 2, 1, f);
    double complex D = cexp(-2.0 * I * M_PI * f * ORC_ARM);
    double complex W = 1.0 - D * D;
    double complex X = W * ((G31 + D * G13) - (G21 + D * G12));
    double complex Y = W * ((G12 + D * G21) - (G32 + D * G23));
    double complex Z = W * ((G23 + D * G32) - (G13 + D * G31));
    out[0] = G12; out[1] = G21; out[2] = G13; out[3] = G31;
    out[4] = G23; out[5] = G32;
    out[6] = X; out[7] = Y; out[8] = Z;
    out[9] = (Z - X) / sqrt(2.0);
    out[10] = (X - 2.0 * Y + Z) / sqrt(6.0);
    out[11] = (X + Y + Z) / sqrt(3.0);
}

/* h_A(f_k), h_E(f_k) and h_T(f_k) for one bin */
static void template_bin(const orc_particle *p, dd f, double amp_scale,
                         double phase0, double complex *hA,
                         double complex *hE, double complex *hT) {
    double fd = dd_to_d(f);
    double t = time_of_freq(p, f);
    double fr = phase_turns_reduced(p, f);
    double complex carrier = cexp(-2.0 * I * M_PI * fr);   /* e^{-i Psi} */
    double amp = (p->waveform == ORC_LINEAR_CHIRP) ? 1.0 : pow(fd, -7.0 / 6.0);
    double complex h = amp_scale * cexp(I * phase0) * amp * carrier;
    if (p->response == ORC_IDENTITY) {
        *hA = h;
        *hE = 0.0;
        *hT = 0.0;
    } else {
        double complex T[12];
        tdi(p, fd, t, T);
        *hA = T[9] * h;
        *hE = T[10] * h;
        *hT = T[11] * h;
    }
}

/* ------------------------------------------------------------------ */
/* compensated summation                                               */
/* ------------------------------------------------------------------ */
typedef struct { double s, c; } nsum;
static void nadd(nsum *a, double x) {
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}
static double nval(const nsum *a) { return a->s + a->c; }

/* ------------------------------------------------------------------ */
/* exported API                                                        */
/* ------------------------------------------------------------------ */

/* Support [k_lo, k_hi] of a particle on the grid f_k = f_first + k df,
 * 0 <= k < K.  Returns ORC_OK, ORC_INVALID (non-physical) or ORC_EMPTY. */
int orc_support(const double *th, int waveform, double f_first, double df,
                int64_t K, double T_obs, int64_t *k_lo, int64_t *k_hi) {
    orc_particle p;
    *k_lo = 0;
    *k_hi = -1;
    if (particle_init(&p, th, waveform, ORC_IDENTITY) != ORC_OK)
        return ORC_INVALID;
    double f0 = th[2];
    double g = ceil((f0 - f_first) / df);
    int64_t k = (g < 0.0) ? 0 : (g > (double)K ? K : (int64_t)g);
    /* exact comparison against the double-double grid frequency */
    while (k > 0 && dd_sub(grid_freq(f_first, df, k - 1), from_d(f0)).hi >= 0.0) --k;
    while (k < K && dd_sub(grid_freq(f_first, df, k), from_d(f0)).hi < 0.0) ++k;
    int64_t lo = k, hi = k - 1;
    /* t(f) and v(f) increase with f, so "in band" holds on a prefix of
     * [lo, K): bisection for its last bin */
    if (k < K && in_band(&p, grid_freq(f_first, df, k), T_obs)) {
        int64_t good = k, bad = K;   /* in_band(good), !in_band(bad) or end */
        while (bad - good > 1) {
            int64_t mid = good + (bad - good) / 2;
            if (in_band(&p, grid_freq(f_first, df, mid), T_obs)) good = mid;
            else bad = mid;
        }
        hi = good;
    }
    *k_lo = lo;
    *k_hi = hi;
    return (hi >= lo) ? ORC_OK : ORC_EMPTY;
}

/* t(f) in seconds; NaN for an invalid particle */
double orc_time_of_freq(const double *th, int waveform, double f) {
    orc_particle p;
    if (particle_init(&p, th, waveform, ORC_IDENTITY) != ORC_OK) return NAN;
    return time_of_freq(&p, from_d(f));
}

/* The PN phase and time split by order at frequency f (pins only):
 * F[j] [turns] and T[j] = dF[j]/df [s] for j = 0..7 (orders 0, 1, 1.5, 2,
 * 2.5, 3, 3.5PN, eccentric).  ORC_INVALID for an invalid particle or a
 * model without a PN phase. */
int orc_pn_terms(const double *th, int waveform, double f, double *Fo,
                 double *To) {
    orc_particle p;
    if (waveform == ORC_LINEAR_CHIRP) return ORC_INVALID;
    if (particle_init(&p, th, waveform, ORC_IDENTITY) != ORC_OK)
        return ORC_INVALID;
    dd F[8], T[8];
    pn_terms(&p, from_d(f), F, T);
    for (int j = 0; j < 8; ++j) {
        Fo[j] = dd_to_d(F[j]);
        To[j] = dd_to_d(T[j]);
    }
    return ORC_OK;
}

/* derived: out[0]=eta, out[1]=M [s], out[2]=t_c [s], out[3]=t_c low part */
int orc_derive(const double *th, int waveform, double *out) {
    orc_particle p;
    int st = particle_init(&p, th, waveform, ORC_IDENTITY);
    out[0] = dd_to_d(p.eta);
    out[1] = dd_to_d(p.Ms);
    out[2] = p.tc.hi;
    out[3] = p.tc.lo;
    return st;
}

/* reduced phase Psi(f)/2pi mod 1 at grid bin k (diagnostic) */
double orc_phase_turns(const double *th, int waveform, double f_first,
                       double df, int64_t k) {
    orc_particle p;
    if (particle_init(&p, th, waveform, ORC_IDENTITY) != ORC_OK) return NAN;
    return phase_turns_reduced(&p, grid_freq(f_first, df, k));
}

/* response diagnostics at frequency f and time t: 12 complex values
 * (6 links, X, Y, Z, A, E, T) interleaved re,im -> out[24]; pos[9] positions */
int orc_response(const double *th, double f, double t, double *out,
                 double *pos) {
    orc_particle p;
    double th2[8];
    memcpy(th2, th, sizeof(th2));
    th2[7] = 0.0;
    if (!(th2[0] > 0.0)) th2[0] = 1.0;   /* response needs only angles */
    if (!(th2[1] >= 1.0)) th2[1] = 1.0;
    if (!(th2[2] > 0.0)) th2[2] = 1e-3;
    particle_init(&p, th2, ORC_LINEAR_CHIRP, ORC_TDI_AE);
    double complex T[12];
    tdi(&p, f, t, T);
    for (int i = 0; i < 12; ++i) {
        out[2 * i] = creal(T[i]);
        out[2 * i + 1] = cimag(T[i]);
    }
    double P[3][3];
    orbit(t, P);
    for (int i = 0; i < 9; ++i) pos[i] = P[i / 3][i % 3];
    return 0;
}

/* template h_A, h_E (and h_T if hT is not NULL) over the whole grid
 * (complex interleaved, zero outside the support).  Returns the support
 * status. */
int orc_template(const double *th, int waveform, int response, double f_first,
                 double df, int64_t K, double T_obs, double amp_scale,
                 double phase0, double *hA, double *hE, double *hT) {
    memset(hA, 0, sizeof(double) * 2 * (size_t)K);
    memset(hE, 0, sizeof(double) * 2 * (size_t)K);
    if (hT) memset(hT, 0, sizeof(double) * 2 * (size_t)K);
    int64_t lo, hi;
    int st = orc_support(th, waveform, f_first, df, K, T_obs, &lo, &hi);
    if (st != ORC_OK) return st;
    orc_particle p;
    particle_init(&p, th, waveform, response);
    for (int64_t k = lo; k <= hi; ++k) {
        double complex a, e, tt;
        template_bin(&p, grid_freq(f_first, df, k), amp_scale, phase0, &a, &e,
                     &tt);
        hA[2 * k] = creal(a);
        hA[2 * k + 1] = cimag(a);
        hE[2 * k] = creal(e);
        hE[2 * k + 1] = cimag(e);
        if (hT) {
            hT[2 * k] = creal(tt);
            hT[2 * k + 1] = cimag(tt);
        }
    }
    return ORC_OK;
}

/* EQUAL_SNR2 boundaries kappa[0..N] from the exact template power on the
 * anchor grid k_lo, k_lo + 1024, ..., k_hi.  hhk[j] = sum_alpha w |h|^2 at
 * support bin k_lo + j.  */
#define ORC_SNR2_STRIDE 1024
#define ORC_SNR2_SNAP 0x1p-20   /* bins; kappa - 2^-20 is exact below 2^32 */
static void snr2_bounds(int64_t lo, int64_t hi, const double *hhk, int N,
                        double *kappa) {
    int64_t nanch = (hi - lo) / ORC_SNR2_STRIDE + 1;
    if ((hi - lo) % ORC_SNR2_STRIDE != 0) ++nanch;
    int64_t *ka = malloc(sizeof(int64_t) * (size_t)nanch);
    double *C = malloc(sizeof(double) * (size_t)nanch);
    for (int64_t a = 0; a < nanch; ++a) {
        int64_t k = lo + a * ORC_SNR2_STRIDE;
        ka[a] = (k > hi) ? hi : k;
    }
    C[0] = 0.0;
    for (int64_t a = 1; a < nanch; ++a)
        C[a] = C[a - 1] + (double)(ka[a] - ka[a - 1]) *
                              (hhk[ka[a - 1] - lo] + hhk[ka[a] - lo]) / 2.0;
    double Clast = C[nanch - 1];
    kappa[0] = (double)lo;
    kappa[N] = (double)(hi + 1);
    int64_t a = 1;   /* targets increase with n: the search only moves up */
    for (int n = 1; n < N; ++n) {
        if (!(Clast > 0.0)) {
            kappa[n] = (double)lo;
            continue;
        }
        double cn = ((double)n * Clast) / (double)N;
        while (a < nanch - 1 && C[a] < cn) ++a;
        kappa[n] = (double)ka[a - 1] + (cn - C[a - 1]) / (C[a] - C[a - 1]) *
                                           (double)(ka[a] - ka[a - 1]);
        kappa[n] -= ORC_SNR2_SNAP;
    }
    free(ka);
    free(C);
}

/*
 * Upsilon_N for P particles.
 *   data: A, E complex interleaved [K]; SA, SE one-sided PSD [K] (SE may be
 *         NULL -> SA);  optional third channel T with its PSD ST (both NULL:
 *         A and E only);  grid f_k = f_first + k df;  T_obs.
 *   params: P x 8 row-major.
 *   stat[P]; optional seg_x[P*N], seg_hh[P*N], kappa[P*(N+1)].
 *   amp_scale, phase0: template multiplied by amp_scale e^{i phase0}
 *   (invariance tests; 1 and 0 otherwise).
 * Invalid particles get stat = -inf; an empty support gives 0.
 */
int orc_eval(double f_first, double df, int64_t K, double T_obs,
             const double *A, const double *E, const double *SA,
             const double *SE, const double *T, const double *ST, int N,
             int mode, int waveform, int response,
             const double *params, int64_t P, double amp_scale, double phase0,
             double *stat, double *seg_x, double *seg_hh, double *kappa,
             int nthreads) {
    if (SE == NULL) SE = SA;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t ip = 0; ip < P; ++ip) {
        const double *th = params + 8 * ip;
        if (seg_x) memset(seg_x + ip * N, 0, sizeof(double) * (size_t)N);
        if (seg_hh) memset(seg_hh + ip * N, 0, sizeof(double) * (size_t)N);
        double *kap = malloc(sizeof(double) * (size_t)(N + 1));
        int64_t lo, hi;
        int st = orc_support(th, waveform, f_first, df, K, T_obs, &lo, &hi);
        if (st == ORC_INVALID) {
            stat[ip] = -INFINITY;
            for (int n = 0; n <= N; ++n) kap[n] = NAN;
        } else if (st == ORC_EMPTY) {
            stat[ip] = 0.0;
            for (int n = 0; n <= N; ++n) kap[n] = NAN;
        } else {
            orc_particle p;
            particle_init(&p, th, waveform, response);
            int64_t S = hi - lo + 1;
            double complex *zk = malloc(sizeof(double complex) * (size_t)S);
            double *hhk = malloc(sizeof(double) * (size_t)S);
            for (int64_t k = lo; k <= hi; ++k) {
                double complex a, e, tt;
                template_bin(&p, grid_freq(f_first, df, k), amp_scale, phase0,
                             &a, &e, &tt);
                double wA = 4.0 * df / SA[k], wE = 4.0 * df / SE[k];
                double complex dA = A[2 * k] + I * A[2 * k + 1];
                double complex dE = E[2 * k] + I * E[2 * k + 1];
                zk[k - lo] = wA * dA * conj(a) + wE * dE * conj(e);
                hhk[k - lo] = wA * (creal(a) * creal(a) + cimag(a) * cimag(a)) +
                              wE * (creal(e) * creal(e) + cimag(e) * cimag(e));
                if (T) {   /* the third channel's terms, added last */
                    double wT = 4.0 * df / ST[k];
                    double complex dT = T[2 * k] + I * T[2 * k + 1];
                    zk[k - lo] += wT * dT * conj(tt);
                    hhk[k - lo] += wT * (creal(tt) * creal(tt) + cimag(tt) * cimag(tt));
                }
            }
            if (mode == ORC_EQUAL_WIDTH) {
                for (int n = 0; n <= N; ++n)
                    kap[n] = (double)((int64_t)n * K / N);
            } else {
                snr2_bounds(lo, hi, hhk, N, kap);
            }
            double ups = 0.0;
            nsum ups_s = {0.0, 0.0};
            int n = 0;
            int64_t k = lo;
            while (n < N && k <= hi) {
                nsum zr = {0, 0}, zi = {0, 0}, hh = {0, 0};
                /* bins of segment n: kappa_n <= k < kappa_{n+1} */
                while (k <= hi && (double)k >= kap[n] && (double)k < kap[n + 1]) {
                    nadd(&zr, creal(zk[k - lo]));
                    nadd(&zi, cimag(zk[k - lo]));
                    nadd(&hh, hhk[k - lo]);
                    ++k;
                }
                double h = nval(&hh);
                double x = hypot(nval(&zr), nval(&zi));
                if (seg_x) seg_x[ip * N + n] = x;
                if (seg_hh) seg_hh[ip * N + n] = h;
                if (h > 0.0) nadd(&ups_s, x * x / h);
                ++n;
            }
            ups = nval(&ups_s);
            stat[ip] = ups;
            free(zk);
            free(hhk);
        }
        if (kappa) memcpy(kappa + ip * (N + 1), kap, sizeof(double) * (size_t)(N + 1));
        free(kap);
    }
    return 0;
}

/* Adds snr * h / sqrt(<h|h>) (one particle) to the data A, E (and T, with
 * PSD ST, if T is not NULL) in place.  Returns the optimal SNR^2 <h|h> of
 * the un-normalised template over the channels given. */
double orc_inject(const double *th, double f_first, double df, int64_t K,
                  double T_obs, const double *SA, const double *SE,
                  const double *ST, double snr, double *A, double *E,
                  double *T) {
    if (SE == NULL) SE = SA;
    double *hA = malloc(sizeof(double) * 2 * (size_t)K);
    double *hE = malloc(sizeof(double) * 2 * (size_t)K);
    double *hT = T ? malloc(sizeof(double) * 2 * (size_t)K) : NULL;
    orc_template(th, ORC_TF2, ORC_TDI_AE, f_first, df, K, T_obs, 1.0, 0.0, hA, hE,
                 hT);
    nsum hh = {0, 0};
    for (int64_t k = 0; k < K; ++k) {
        nadd(&hh, 4.0 * df / SA[k] * (hA[2 * k] * hA[2 * k] + hA[2 * k + 1] * hA[2 * k + 1]));
        nadd(&hh, 4.0 * df / SE[k] * (hE[2 * k] * hE[2 * k] + hE[2 * k + 1] * hE[2 * k + 1]));
        if (T)
            nadd(&hh, 4.0 * df / ST[k] * (hT[2 * k] * hT[2 * k] + hT[2 * k + 1] * hT[2 * k + 1]));
    }
    double h2 = nval(&hh);
    double s = (h2 > 0.0) ? snr / sqrt(h2) : 0.0;
    for (int64_t i = 0; i < 2 * K; ++i) {
        A[i] += s * hA[i];
        E[i] += s * hE[i];
        if (T) T[i] += s * hT[i];
    }
    free(hA);
    free(hE);
    free(hT);
    return h2;
}
