/*
 * lboracle.c -- plain, slow, FP64 CPU oracle for the tracer-box lattice
 * Boltzmann method of Lee, Duenweg and Schumacher (arXiv:0809.4958) with a
 * bead-spring chain coupled by Stokes friction.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * includes this file; it shares no code, header, table or constant generator
 * with the CUDA path.  It is built as its own shared object and driven from
 * Python (oracle/__init__.py) by the tests and by the CPU-baseline leg of the
 * benchmark.
 *
 * What it computes, in the order the method takes its steps:
 *   - D3Q19 lattice, BGK collision (Sec. 3: "standard D3Q19 model"; the
 *     collision operator is not printed, single-relaxation BGK is the reading),
 *     second-order equilibrium, Guo forcing for body and bead forces.
 *   - Initial condition: local equilibrium with the prescribed velocity on
 *     every site at t = 0 (Sec. 2).
 *   - Boundary condition: at later times the sites of the outer layer are set
 *     to their local equilibrium with the prescribed boundary velocity (Sec. 2),
 *     interpolated in time between coarse samples (Sec. 3, Eq. 1 and the
 *     interpolation remark after it).
 *   - Bead-spring (FENE) chain coupled to the fluid by a Stokes friction
 *     coefficient (Sec. 1, hybrid LB-MD method of Ahlrichs and Duenweg) with
 *     the chain centre of mass pinned at the box centre (Sec. 2).
 *   - The synthetic coarse flow that stands in for the DNS sub-volume record
 *     (a sum of Fourier modes with a Kolmogorov spectrum).
 *   - Philox4x32-10 (Salmon et al., SC'11) for the bead noise.
 *
 * Everything is written for clarity, site by site, with no blocking or fusion.
 * OpenMP only splits the z loop of the lattice sweep; the arithmetic of each
 * site does not depend on it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define Q 19

/* D3Q19 velocities: rest, 6 face neighbours (+x,-x,+y,-y,+z,-z), 12 edge
 * neighbours.  Opposite directions sit in adjacent slots (1<->2, 3<->4, ...). */
static const int CV[Q][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

static const double WV[Q] = {
    1.0 / 3.0,
    1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

static const double CS2 = 1.0 / 3.0; /* speed of sound squared */

enum {
    ORC_OK = 0,
    ORC_ERR_ARG = 1,
    ORC_ERR_FENE = 2,     /* a bond reached the FENE maximum extension R0 */
    ORC_ERR_BEAD_OOB = 3, /* a bead's interpolation stencil left the interior */
    ORC_ERR_SAMPLES = 4   /* the boundary needs a coarse sample that was not given */
};

enum { ORC_TIME_LINEAR = 0, ORC_TIME_HERMITE = 1, ORC_TIME_MLP = 2 };
enum { ORC_STORE_F64 = 0, ORC_STORE_F16 = 2, ORC_STORE_BF16 = 3 };

typedef struct {
    int32_t E;           /* sites per axis */
    int32_t periodic[3]; /* per axis: 1 periodic, 0 both faces carry the velocity condition */
    double tau;          /* BGK relaxation time, nu = cs^2 (tau - 1/2) */
    double rho_b;        /* density of the boundary equilibrium */
    double accel[3];     /* uniform body acceleration a (force density rho a) */
    int32_t time_interp; /* ORC_TIME_* */
    int32_t K;           /* LB steps per coarse sample interval */
    int32_t storage;     /* ORC_STORE_*: emulate 16-bit storage of f_i - w_i */
    int32_t zoom;        /* z = coarse grid spacing / LB spacing (Sec. 3) */
} orc_box;

/* points per axis of the coarse grid of a box: coarse point P sits at site
 * P z, from site 0 until the grid covers site E - 1 (the last coarse cell may
 * reach past the box when z does not divide E - 1) */
static int coarse_points_of(int E, int z) { return z > 1 ? (E - 1 + z - 1) / z + 1 : E; }
static int coarse_points(const orc_box *b) { return coarse_points_of(b->E, b->zoom); }
static int zoom_of(const orc_box *b) { return b->zoom > 1 ? b->zoom : 1; }

typedef struct {
    int32_t nbeads;
    int32_t n_md;    /* MD substeps per LB step */
    int32_t pin_com; /* 0 off, 1 position, 2 position and velocity */
    int32_t pad;
    double k_fene, R0, zeta, mass, kT;
    double eps, sigma; /* WCA repulsion between all bead pairs (eps = 0: FENE only) */
    double f_ext[3]; /* constant external force on every bead (tests only) */
    uint64_t seed;
    uint64_t box_id;
} orc_chain;

/* ------------------------------------------------------------------ */
/* lattice constants, exported so tests can look at them              */

void orc_lattice(int32_t *c, double *w)
{
    for (int i = 0; i < Q; i++) {
        for (int a = 0; a < 3; a++) c[3 * i + a] = CV[i][a];
        w[i] = WV[i];
    }
}

/* Second-order equilibrium f_i^eq = w_i rho (1 + c.u/cs2 + (c.u)^2/(2 cs2^2) - u.u/(2 cs2)). */
void orc_equilibrium(double rho, const double u[3], double feq[Q])
{
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < Q; i++) {
        double cu = CV[i][0] * u[0] + CV[i][1] * u[1] + CV[i][2] * u[2];
        feq[i] = WV[i] * rho * (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
    }
}

/* ------------------------------------------------------------------ */
/* IEEE binary16 and bfloat16 round-to-nearest-even, for emulating     */
/* 16-bit storage of the deviations f_i - w_i.                          */

/* Round x to the nearest binary16 value (ties to even) and return it as a double. */
double orc_round_f16(double x)
{
    if (x != x) return x;
    double ax = fabs(x);
    if (ax >= 65520.0) return x > 0 ? INFINITY : -INFINITY; /* beyond max + half ulp */
    int e;
    frexp(ax, &e); /* ax = m * 2^e, m in [0.5, 1) */
    int exp_unbiased = e - 1;          /* ax in [2^(e-1), 2^e) */
    if (exp_unbiased < -14) exp_unbiased = -14; /* subnormal range has a fixed quantum */
    double quantum = ldexp(1.0, exp_unbiased - 10);
    double r = nearbyint(ax / quantum) * quantum; /* default rounding mode: ties to even */
    return x < 0 ? -r : r;
}

/* Round x to the nearest bfloat16 value (8-bit significand, ties to even). */
double orc_round_bf16(double x)
{
    if (x != x) return x;
    double ax = fabs(x);
    if (ax == 0.0) return x;
    int e;
    frexp(ax, &e);
    int exp_unbiased = e - 1;
    if (exp_unbiased < -126) exp_unbiased = -126;
    double quantum = ldexp(1.0, exp_unbiased - 7);
    double r = nearbyint(ax / quantum) * quantum;
    if (r > 3.3895313892515355e38) r = INFINITY;
    return x < 0 ? -r : r;
}

static double store_round(int storage, double d)
{
    if (storage == ORC_STORE_F16) return orc_round_f16(d);
    if (storage == ORC_STORE_BF16) return orc_round_bf16(d);
    return d;
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,   */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds of */
/* two 32x32->64 multiplications with the key bumped by two Weyl        */
/* constants between rounds.                                            */

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t p0 = (uint64_t)M0 * x0, p1 = (uint64_t)M1 * x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Unit-variance uniform number on [-sqrt3, sqrt3) from a 32-bit word:
 * u = v 2^-32 (exact in double), xi = sqrt3 (2u - 1). */
static double uniform_unit_variance(uint32_t v)
{
    double u01 = (double)v * (1.0 / 4294967296.0); /* 2^-32 */
    return sqrt(3.0) * (2.0 * u01 - 1.0);
}

/* ------------------------------------------------------------------ */
/* site helpers                                                       */

static inline long site_index(int E, int x, int y, int z) { return ((long)z * E + y) * E + x; }

static inline int wrap(int v, int E) { return ((v % E) + E) % E; }

/* 1 if the site lies on the outer layer of an axis whose faces carry the velocity condition. */
static int is_boundary_site(const orc_box *b, int x, int y, int z)
{
    int E = b->E;
    if (!b->periodic[0] && (x == 0 || x == E - 1)) return 1;
    if (!b->periodic[1] && (y == 0 || y == E - 1)) return 1;
    if (!b->periodic[2] && (z == 0 || z == E - 1)) return 1;
    return 0;
}

/* The face that owns a boundary site: the first velocity face containing it,
 * in the order x-, x+, y-, y+, z-, z+.  Also returns the in-face coordinates
 * (p, q): (y, z) on x faces, (x, z) on y faces, (x, y) on z faces. */
static int owning_face(const orc_box *b, int x, int y, int z, int *p, int *q)
{
    int E = b->E;
    if (!b->periodic[0] && x == 0) { *p = y; *q = z; return 0; }
    if (!b->periodic[0] && x == E - 1) { *p = y; *q = z; return 1; }
    if (!b->periodic[1] && y == 0) { *p = x; *q = z; return 2; }
    if (!b->periodic[1] && y == E - 1) { *p = x; *q = z; return 3; }
    if (!b->periodic[2] && z == 0) { *p = x; *q = y; return 4; }
    if (!b->periodic[2] && z == E - 1) { *p = x; *q = y; return 5; }
    return -1;
}

/* Populations arriving at site (x,y,z) by streaming: f_i(x) = A_i(x - c_i),
 * wrapped on periodic axes.  The caller only asks for non-boundary sites, so
 * on velocity axes x - c_i stays inside the box. */
static void pulled(const orc_box *b, const double *A, int x, int y, int z, double fi[Q])
{
    int E = b->E;
    long n3 = (long)E * E * E;
    for (int i = 0; i < Q; i++) {
        int xs = x - CV[i][0], ys = y - CV[i][1], zs = z - CV[i][2];
        if (b->periodic[0]) xs = wrap(xs, E);
        if (b->periodic[1]) ys = wrap(ys, E);
        if (b->periodic[2]) zs = wrap(zs, E);
        fi[i] = A[i * n3 + site_index(E, xs, ys, zs)];
    }
}

static void moments(const double fi[Q], double *rho, double j[3])
{
    *rho = 0.0;
    j[0] = j[1] = j[2] = 0.0;
    for (int i = 0; i < Q; i++) {
        *rho += fi[i];
        for (int a = 0; a < 3; a++) j[a] += CV[i][a] * fi[i];
    }
}

/* ------------------------------------------------------------------ */
/* time interpolation of the coarse boundary samples                  */

/* Coarse samples: samples[j][face][comp][q][p], sample j taken at t = j K.
 * Boundary velocity at time t = n + 1 (the end of step n -> n+1), t in
 * (jK, (j+1)K] with j = floor(n / K):
 *   linear:  (1-th) U_j + th U_{j+1}, th = (t - jK)/K
 *   Hermite: cubic Hermite with Catmull-Rom tangents m_j = (U_{j+1}-U_{j-1})/2,
 *            one-sided m_0 = U_1 - U_0 on the first interval
 *   MLP:     Hermite plus a learned residual r[face][comp][s-1][q][p],
 *            s = t - jK in 1..K, supplied by the caller for interval j.
 * The samples live on the coarse face grid ([6][3][Ec][Ec], point P at site
 * P z).  With zoom z > 1 the velocity at a
 * site is the bilinear interpolation, within the face, of the time-interpolated
 * velocities at the four surrounding coarse points (Sec. 3: bilinear in space
 * between neighbouring grid points, linear in time). */
static int coarse_velocity(const orc_box *b, const double *samples, long nsamples, long n, int f, int P, int Qc,
                           double u[3])
{
    int K = b->K, Ec = coarse_points(b);
    long j = n / K;
    int s = (int)(n + 1 - j * K);
    double th = (double)s / (double)K;
    long face_stride = 3L * Ec * Ec;
#define U_AT(jj, c) samples[((long)(jj) * 6 + f) * face_stride + (long)(c) * Ec * Ec + (long)Qc * Ec + P]
    if (b->time_interp == ORC_TIME_LINEAR) {
        if (j + 1 >= nsamples) return ORC_ERR_SAMPLES;
        for (int c = 0; c < 3; c++) u[c] = (1.0 - th) * U_AT(j, c) + th * U_AT(j + 1, c);
        return ORC_OK;
    }
    if (j + 2 >= nsamples) return ORC_ERR_SAMPLES;
    double h00 = 2 * th * th * th - 3 * th * th + 1;
    double h10 = th * th * th - 2 * th * th + th;
    double h01 = -2 * th * th * th + 3 * th * th;
    double h11 = th * th * th - th * th;
    for (int c = 0; c < 3; c++) {
        double u0 = U_AT(j, c), u1 = U_AT(j + 1, c), u2 = U_AT(j + 2, c);
        double m0 = (j >= 1) ? 0.5 * (u1 - U_AT(j - 1, c)) : (u1 - u0);
        double m1 = 0.5 * (u2 - u0);
        u[c] = h00 * u0 + h10 * m0 + h01 * u1 + h11 * m1;
    }
#undef U_AT
    return ORC_OK;
}

static int face_velocity(const orc_box *b, const double *samples, long nsamples,
                         const double *resid, long n, int f, int p, int q, double u[3])
{
    int E = b->E, K = b->K, z = zoom_of(b);
    if (z == 1) {
        int e = coarse_velocity(b, samples, nsamples, n, f, p, q, u);
        if (e) return e;
    } else {
        /* coarse cell (P0, Q0) holding the site and the site's fractions in it */
        int P0 = p / z, Q0 = q / z, Ec = coarse_points(b);
        int P1 = P0 + 1 < Ec ? P0 + 1 : P0, Q1 = Q0 + 1 < Ec ? Q0 + 1 : Q0;
        double fp = (double)(p - P0 * z) / z, fq = (double)(q - Q0 * z) / z;
        double u00[3], u10[3], u01[3], u11[3];
        int e = coarse_velocity(b, samples, nsamples, n, f, P0, Q0, u00);
        if (!e) e = coarse_velocity(b, samples, nsamples, n, f, P1, Q0, u10);
        if (!e) e = coarse_velocity(b, samples, nsamples, n, f, P0, Q1, u01);
        if (!e) e = coarse_velocity(b, samples, nsamples, n, f, P1, Q1, u11);
        if (e) return e;
        for (int c = 0; c < 3; c++)
            u[c] = (1.0 - fq) * ((1.0 - fp) * u00[c] + fp * u10[c]) + fq * ((1.0 - fp) * u01[c] + fp * u11[c]);
    }
    if (b->time_interp == ORC_TIME_MLP && resid && z == 1) {
        int s = (int)(n + 1 - (n / K) * K);
        for (int c = 0; c < 3; c++) u[c] += resid[(((long)f * 3 + c) * K + (s - 1)) * E * E + (long)q * E + p];
    }
    return ORC_OK;
}

/* Exported for tests: boundary velocity of face f, site (p, q), at time n + 1. */
int orc_face_velocity(const orc_box *b, const double *samples, long nsamples, const double *resid,
                      long n, int f, int p, int q, double u[3])
{
    return face_velocity(b, samples, nsamples, resid, n, f, p, q, u);
}

/* ------------------------------------------------------------------ */
/* initial condition: local equilibrium with rho = 1 and u0 on every site */

/* u0: the field on the coarse grid, [3][Ec][Ec][Ec] (the sites themselves when
 * z = 1); with z > 1 each site takes the trilinear interpolation of the eight
 * surrounding coarse points (Sec. 2: the initial field interpolated linearly
 * from the DNS grid). */
void orc_init(const orc_box *b, const double *u0 /* [3][Ec^3] */, double *f /* [19][E^3] */)
{
    int E = b->E, z = zoom_of(b), Ec = coarse_points(b);
    long n3 = (long)E * E * E, c3 = (long)Ec * Ec * Ec;
    for (int zz = 0; zz < E; zz++)
        for (int y = 0; y < E; y++)
            for (int x = 0; x < E; x++) {
                long s = site_index(E, x, y, zz);
                double u[3], feq[Q];
                if (z == 1) {
                    for (int c = 0; c < 3; c++) u[c] = u0[c * c3 + s];
                } else {
                    int i0[3] = {x / z, y / z, zz / z}, i1[3];
                    double fr[3];
                    int xyz[3] = {x, y, zz};
                    for (int a = 0; a < 3; a++) {
                        i1[a] = i0[a] + 1 < Ec ? i0[a] + 1 : i0[a];
                        fr[a] = (double)(xyz[a] - i0[a] * z) / z;
                    }
                    for (int c = 0; c < 3; c++) {
                        double acc = 0.0;
                        for (int k = 0; k < 8; k++) {
                            int X = (k & 1) ? i1[0] : i0[0], Y = (k & 2) ? i1[1] : i0[1], Z = (k & 4) ? i1[2] : i0[2];
                            double w = ((k & 1) ? fr[0] : 1.0 - fr[0]) * ((k & 2) ? fr[1] : 1.0 - fr[1]) *
                                       ((k & 4) ? fr[2] : 1.0 - fr[2]);
                            acc += w * u0[c * c3 + ((long)Z * Ec + Y) * Ec + X];
                        }
                        u[c] = acc;
                    }
                }
                orc_equilibrium(1.0, u, feq);
                for (int i = 0; i < Q; i++) f[i * n3 + s] = WV[i] + store_round(b->storage, feq[i] - WV[i]);
            }
}

/* ------------------------------------------------------------------ */
/* fluid velocity seen by a bead                                      */

/* Velocity of the pulled populations at an interior site, with the half
 * body-force shift: u = (j + rho a / 2) / rho. */
static void site_velocity(const orc_box *b, const double *A, int x, int y, int z, double u[3])
{
    double fi[Q], rho, j[3];
    pulled(b, A, x, y, z, fi);
    moments(fi, &rho, j);
    for (int a = 0; a < 3; a++) u[a] = (j[a] + 0.5 * rho * b->accel[a]) / rho;
}

/* Trilinear stencil of a point R: base cell corner i0 = floor(R) and the eight
 * weights w_c = prod_a (c_a ? d_a : 1 - d_a), d = R - i0.  Corner index
 * c = cx + 2 cy + 4 cz.  Returns ORC_ERR_BEAD_OOB if, on a velocity axis, the
 * cell is not inside the interior [1, E-2]. */
static int trilinear_stencil(const orc_box *b, const double R[3], int base[3], double w[8])
{
    int E = b->E;
    double d[3];
    for (int a = 0; a < 3; a++) {
        double fl = floor(R[a]);
        d[a] = R[a] - fl;
        long i0 = (long)fl;
        if (!b->periodic[a]) {
            if (i0 < 1 || i0 + 1 > E - 2) return ORC_ERR_BEAD_OOB;
            base[a] = (int)i0;
        } else {
            base[a] = (int)(((i0 % E) + E) % E);
        }
    }
    for (int c = 0; c < 8; c++) {
        int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
        w[c] = (cx ? d[0] : 1.0 - d[0]) * (cy ? d[1] : 1.0 - d[1]) * (cz ? d[2] : 1.0 - d[2]);
    }
    return ORC_OK;
}

static void corner_site(const orc_box *b, const int base[3], int c, int xyz[3])
{
    int off[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
    for (int a = 0; a < 3; a++) {
        int v = base[a] + off[a];
        xyz[a] = b->periodic[a] ? wrap(v, b->E) : v;
    }
}

/* Exported for tests: trilinear interpolation of the fluid velocity at R. */
int orc_interp_velocity(const orc_box *b, const double *A, const double R[3], double u[3])
{
    int base[3];
    double w[8];
    int st = trilinear_stencil(b, R, base, w);
    if (st) return st;
    u[0] = u[1] = u[2] = 0.0;
    for (int c = 0; c < 8; c++) {
        int s[3];
        double uc[3];
        corner_site(b, base, c, s);
        site_velocity(b, A, s[0], s[1], s[2], uc);
        for (int a = 0; a < 3; a++) u[a] += w[c] * uc[a];
    }
    return ORC_OK;
}

/* Kremer-Grest bead-spring forces on every bead of a linear chain (the chain
 * model of the Ahlrichs-Duenweg hybrid method the paper builds on, Sec. 1):
 *   FENE per bond, U(r) = -k R0^2/2 ln(1 - r^2/R0^2): force on bead b+1 is
 *     -k r / (1 - r^2/R0^2) with r = R_{b+1} - R_b, the opposite on bead b;
 *   WCA between every pair, U(r) = 4 eps ((s/r)^12 - (s/r)^6) + eps for
 *     r < 2^(1/6) s: force on bead j is 24 eps (2 (s/r)^12 - (s/r)^6) r / r^2
 *     with r = R_j - R_i, the opposite on bead i.
 * Bond terms are added first, then pair terms in increasing partner order. */
int orc_chain_forces(int nbeads, double k, double R0, double eps, double sigma, const double *R, double *F)
{
    for (int i = 0; i < 3 * nbeads; i++) F[i] = 0.0;
    for (int bb = 0; bb + 1 < nbeads; bb++) {
        double r[3], r2 = 0.0;
        for (int a = 0; a < 3; a++) {
            r[a] = R[3 * (bb + 1) + a] - R[3 * bb + a];
            r2 += r[a] * r[a];
        }
        if (r2 >= R0 * R0) return ORC_ERR_FENE;
        double fac = k / (1.0 - r2 / (R0 * R0));
        for (int a = 0; a < 3; a++) {
            F[3 * bb + a] += fac * r[a];
            F[3 * (bb + 1) + a] -= fac * r[a];
        }
    }
    if (eps > 0.0) {
        double rc2 = cbrt(2.0) * sigma * sigma; /* (2^(1/6) sigma)^2 */
        for (int i = 0; i < nbeads; i++)
            for (int j = i + 1; j < nbeads; j++) {
                double r[3], r2 = 0.0;
                for (int a = 0; a < 3; a++) {
                    r[a] = R[3 * j + a] - R[3 * i + a];
                    r2 += r[a] * r[a];
                }
                if (r2 >= rc2) continue;
                double s2 = sigma * sigma / r2, s6 = s2 * s2 * s2;
                double fac = 24.0 * eps * (2.0 * s6 * s6 - s6) / r2;
                for (int a = 0; a < 3; a++) {
                    F[3 * i + a] -= fac * r[a];
                    F[3 * j + a] += fac * r[a];
                }
            }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* one coupling step of the chain (reads the post-collision state A)   */

/* Runs the chain over one LB step n:
 *   1. fluid velocity at each bead from the pulled populations of A,
 *      trilinear in the start-of-step position;
 *   2. n_md substeps of symplectic Euler (V += dt F / m, R += dt V), with
 *      FENE + WCA + friction -zeta (V - u) + noise sqrt(2 kT zeta / dt) xi
 *      + f_ext, u frozen over the step;
 *   3. centre of mass pinned at the box centre ((E-1)/2 on each axis);
 *   4. the momentum the beads gave to the fluid, -sum (F_fric + F_noise) dt,
 *      spread with the start-of-step trilinear weights into g[3][E^3]
 *      (force density, accumulated in bead order; caller zeroes g).
 * Noise: xi_a from Philox4x32-10, counter (n mod 2^32, substep, bead, box_id),
 * key (low and high 32 bits of seed), word a, mapped to a uniform number with
 * unit variance. */
int orc_chain_couple(const orc_box *b, const orc_chain *ch, const double *A, long n,
                     double *pos, double *vel, double *g)
{
    int N = ch->nbeads, E = b->E;
    long n3 = (long)E * E * E;
    if (N <= 0) return ORC_OK;
    int *base = (int *)malloc(sizeof(int) * 3 * N);
    double *wts = (double *)malloc(sizeof(double) * 8 * N);
    double *uR = (double *)malloc(sizeof(double) * 3 * N);
    double *P = (double *)calloc(3 * N, sizeof(double));
    double *F = (double *)malloc(sizeof(double) * 3 * N);
    int st = ORC_OK;

    /* 1. fluid velocity at the beads */
    for (int bb = 0; bb < N && !st; bb++) {
        st = trilinear_stencil(b, &pos[3 * bb], &base[3 * bb], &wts[8 * bb]);
        if (st) break;
        uR[3 * bb] = uR[3 * bb + 1] = uR[3 * bb + 2] = 0.0;
        for (int c = 0; c < 8; c++) {
            int s[3];
            double uc[3];
            corner_site(b, &base[3 * bb], c, s);
            site_velocity(b, A, s[0], s[1], s[2], uc);
            for (int a = 0; a < 3; a++) uR[3 * bb + a] += wts[8 * bb + c] * uc[a];
        }
    }

    /* 2. MD substeps */
    double dt = 1.0 / ch->n_md;
    double noise_amp = ch->kT > 0.0 ? sqrt(2.0 * ch->kT * ch->zeta / dt) : 0.0;
    for (int sub = 0; sub < ch->n_md && !st; sub++) {
        st = orc_chain_forces(N, ch->k_fene, ch->R0, ch->eps, ch->sigma, pos, F);
        if (st) break;
        for (int bb = 0; bb < N; bb++) {
            double xi[3] = {0.0, 0.0, 0.0};
            if (noise_amp > 0.0) {
                uint32_t ctr[4] = {(uint32_t)n, (uint32_t)sub, (uint32_t)bb, (uint32_t)ch->box_id};
                uint32_t key[2] = {(uint32_t)ch->seed, (uint32_t)(ch->seed >> 32)};
                uint32_t r[4];
                orc_philox4x32_10(ctr, key, r);
                for (int a = 0; a < 3; a++) xi[a] = uniform_unit_variance(r[a]);
            }
            for (int a = 0; a < 3; a++) {
                double ffric = -ch->zeta * (vel[3 * bb + a] - uR[3 * bb + a]);
                double fnoise = noise_amp * xi[a];
                double ftot = F[3 * bb + a] + ffric + fnoise + ch->f_ext[a];
                vel[3 * bb + a] += dt / ch->mass * ftot;
                pos[3 * bb + a] += dt * vel[3 * bb + a];
                P[3 * bb + a] -= (ffric + fnoise) * dt;
            }
        }
    }

    /* 3. centre of mass pinned at the box centre */
    if (!st && ch->pin_com >= 1) {
        double com[3] = {0, 0, 0}, vcm[3] = {0, 0, 0};
        for (int bb = 0; bb < N; bb++)
            for (int a = 0; a < 3; a++) {
                com[a] += pos[3 * bb + a];
                vcm[a] += vel[3 * bb + a];
            }
        double centre = 0.5 * (E - 1);
        for (int a = 0; a < 3; a++) {
            com[a] /= N;
            vcm[a] /= N;
        }
        for (int bb = 0; bb < N; bb++)
            for (int a = 0; a < 3; a++) {
                pos[3 * bb + a] += centre - com[a];
                if (ch->pin_com >= 2) vel[3 * bb + a] -= vcm[a];
            }
    }

    /* 4. momentum to the fluid, spread with the start-of-step weights */
    if (!st) {
        for (int bb = 0; bb < N; bb++)
            for (int c = 0; c < 8; c++) {
                int s[3];
                corner_site(b, &base[3 * bb], c, s);
                long idx = site_index(E, s[0], s[1], s[2]);
                for (int a = 0; a < 3; a++) g[a * n3 + idx] += wts[8 * bb + c] * P[3 * bb + a];
            }
    }
    free(base); free(wts); free(uR); free(P); free(F);
    return st;
}

/* ------------------------------------------------------------------ */
/* one LB step n -> n+1                                               */

/* A: post-collision populations at step n (boundary sites hold the
 * equilibrium of t = n).  Writes the post-collision populations of step
 * n + 1 into B.  g: scratch [3][E^3] for the bead force density. */
int orc_step(const orc_box *b, const orc_chain *ch, const double *A, double *B, double *g,
             const double *samples, long nsamples, const double *resid, long n,
             double *pos, double *vel)
{
    int E = b->E;
    long n3 = (long)E * E * E;
    int st = ORC_OK;
    memset(g, 0, sizeof(double) * 3 * n3);
    if (ch && ch->nbeads > 0) {
        st = orc_chain_couple(b, ch, A, n, pos, vel, g);
        if (st) return st;
    }
    double tau = b->tau;
    int serr = ORC_OK;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < E; z++) {
        for (int y = 0; y < E; y++) {
            for (int x = 0; x < E; x++) {
                long s = site_index(E, x, y, z);
                double out[Q];
                if (is_boundary_site(b, x, y, z)) {
                    int p, q;
                    int f = owning_face(b, x, y, z, &p, &q);
                    double ub[3];
                    int e = face_velocity(b, samples, nsamples, resid, n, f, p, q, ub);
                    if (e) {
#pragma omp critical
                        serr = e;
                        ub[0] = ub[1] = ub[2] = 0.0;
                    }
                    orc_equilibrium(b->rho_b, ub, out);
                } else {
                    double fi[Q], rho, j[3], F[3], u[3], feq[Q];
                    pulled(b, A, x, y, z, fi);
                    moments(fi, &rho, j);
                    for (int a = 0; a < 3; a++) {
                        F[a] = rho * b->accel[a] + g[a * n3 + s];
                        u[a] = (j[a] + 0.5 * F[a]) / rho;
                    }
                    orc_equilibrium(rho, u, feq);
                    for (int i = 0; i < Q; i++) {
                        /* Guo forcing: (1 - 1/(2 tau)) w_i [(c_i - u)/cs2 + (c_i.u) c_i/cs2^2] . F */
                        double cu = CV[i][0] * u[0] + CV[i][1] * u[1] + CV[i][2] * u[2];
                        double src = 0.0;
                        for (int a = 0; a < 3; a++)
                            src += ((CV[i][a] - u[a]) / CS2 + cu * CV[i][a] / (CS2 * CS2)) * F[a];
                        src *= (1.0 - 0.5 / tau) * WV[i];
                        out[i] = fi[i] - (fi[i] - feq[i]) / tau + src;
                    }
                }
                for (int i = 0; i < Q; i++) B[i * n3 + s] = WV[i] + store_round(b->storage, out[i] - WV[i]);
            }
        }
    }
    return serr;
}

/* Runs nsteps steps starting at step n0; the result ends in f.  tmp and g are
 * scratch of 19 E^3 and 3 E^3 doubles.  resid (MLP mode) holds one residual
 * block per coarse interval: resid[j][6][3][K][E][E]. */
int orc_run(const orc_box *b, const orc_chain *ch, double *f, double *tmp, double *g,
            const double *samples, long nsamples, const double *resid, long n0, long nsteps,
            double *pos, double *vel)
{
    int E = b->E;
    long n3 = (long)E * E * E;
    long rstride = 6L * 3 * b->K * E * E;
    for (long n = n0; n < n0 + nsteps; n++) {
        const double *r = resid ? resid + (n / b->K) * rstride : NULL;
        int st = orc_step(b, ch, f, tmp, g, samples, nsamples, r, n, pos, vel);
        if (st) return st;
        memcpy(f, tmp, sizeof(double) * Q * n3);
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* observables                                                        */

/* Density and velocity field: on boundary sites the moments of the stored
 * equilibrium, elsewhere the moments of the pulled populations with
 * u = (j + rho a / 2) / rho. */
void orc_fields(const orc_box *b, const double *A, double *rho_out /* [E^3] */, double *u_out /* [3][E^3] */)
{
    int E = b->E;
    long n3 = (long)E * E * E;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < E; z++)
        for (int y = 0; y < E; y++)
            for (int x = 0; x < E; x++) {
                long s = site_index(E, x, y, z);
                double fi[Q], rho, j[3];
                if (is_boundary_site(b, x, y, z)) {
                    for (int i = 0; i < Q; i++) fi[i] = A[i * n3 + s];
                    moments(fi, &rho, j);
                    for (int a = 0; a < 3; a++) u_out[a * n3 + s] = j[a] / rho;
                } else {
                    pulled(b, A, x, y, z, fi);
                    moments(fi, &rho, j);
                    for (int a = 0; a < 3; a++) u_out[a * n3 + s] = (j[a] + 0.5 * rho * b->accel[a]) / rho;
                }
                rho_out[s] = rho;
            }
}

/* Mass sum f_i, momentum sum c_i f_i over all sites of A, and the bead
 * momentum m sum V (out[4..6]). */
void orc_conservation(const orc_box *b, const double *A, int nbeads, double mass, const double *vel,
                      double out[7])
{
    int E = b->E;
    long n3 = (long)E * E * E;
    for (int k = 0; k < 7; k++) out[k] = 0.0;
    for (int i = 0; i < Q; i++)
        for (long s = 0; s < n3; s++) {
            double v = A[i * n3 + s];
            out[0] += v;
            for (int a = 0; a < 3; a++) out[1 + a] += CV[i][a] * v;
        }
    for (int bb = 0; bb < nbeads; bb++)
        for (int a = 0; a < 3; a++) out[4 + a] += mass * vel[3 * bb + a];
}

/* ------------------------------------------------------------------ */
/* synthetic coarse flow (stands in for the DNS sub-volume record)      */

/* u(x, t) = sum_m amp_m cos(kvec_m . (x - xc) + omega_m t + phi_m), with
 * kvec_m = (2 pi k_m / E) khat_m and amp_m = S A_m e_m (e_m perpendicular to
 * khat_m, so the field is divergence free).  pts: [npts][3], out: [npts][3]. */
void orc_field(const double *kvec, const double *amp, const double *omega, const double *phi, int M,
               const double xc[3], const double *pts, long npts, double t, double *out)
{
#pragma omp parallel for schedule(static)
    for (long p = 0; p < npts; p++) {
        double u[3] = {0.0, 0.0, 0.0};
        for (int m = 0; m < M; m++) {
            double ph = kvec[3 * m] * (pts[3 * p] - xc[0]) + kvec[3 * m + 1] * (pts[3 * p + 1] - xc[1]) +
                        kvec[3 * m + 2] * (pts[3 * p + 2] - xc[2]) + omega[m] * t + phi[m];
            double cph = cos(ph);
            for (int a = 0; a < 3; a++) u[a] += amp[3 * m + a] * cph;
        }
        for (int a = 0; a < 3; a++) out[3 * p + a] = u[a];
    }
}

/* Coarse face samples j0 .. j0+nsamp-1, taken at t = j K, evaluated at the
 * coarse face points (site P zoom, Ec points per side): out[j][face][comp][Q][P]. */
void orc_face_samples(const double *kvec, const double *amp, const double *omega, const double *phi,
                      int M, int E, int zoom, int K, long j0, long nsamp, double *out)
{
    double xc[3] = {0.5 * (E - 1), 0.5 * (E - 1), 0.5 * (E - 1)};
    int z = zoom > 1 ? zoom : 1, Ec = coarse_points_of(E, z);
    long ns = (long)Ec * Ec;
    double *pts = (double *)malloc(sizeof(double) * 3 * ns);
    double *val = (double *)malloc(sizeof(double) * 3 * ns);
    for (long j = 0; j < nsamp; j++) {
        double t = (double)((j0 + j) * K);
        for (int f = 0; f < 6; f++) {
            int axis = f / 2;
            int fixed = (f % 2) ? E - 1 : 0;
            for (int q = 0; q < Ec; q++)
                for (int p = 0; p < Ec; p++) {
                    double *P = &pts[3 * ((long)q * Ec + p)];
                    double pp = (double)p * z, qq = (double)q * z;
                    if (axis == 0) { P[0] = fixed; P[1] = pp; P[2] = qq; }
                    else if (axis == 1) { P[0] = pp; P[1] = fixed; P[2] = qq; }
                    else { P[0] = pp; P[1] = qq; P[2] = fixed; }
                }
            orc_field(kvec, amp, omega, phi, M, xc, pts, ns, t, val);
            for (int c = 0; c < 3; c++)
                for (long s = 0; s < ns; s++) out[((j * 6 + f) * 3 + c) * ns + s] = val[3 * s + c];
        }
    }
    free(pts);
    free(val);
}

/* Field at time t on the coarse grid (every zoom-th site, Ec points per
 * axis; every site when zoom = 1): out[comp][Z][Y][X]. */
void orc_volume_field(const double *kvec, const double *amp, const double *omega, const double *phi,
                      int M, int E, int zoom, double t, double *out)
{
    double xc[3] = {0.5 * (E - 1), 0.5 * (E - 1), 0.5 * (E - 1)};
    int zm = zoom > 1 ? zoom : 1, Ec = coarse_points_of(E, zm);
    long n3 = (long)Ec * Ec * Ec;
    double *pts = (double *)malloc(sizeof(double) * 3 * n3);
    double *val = (double *)malloc(sizeof(double) * 3 * n3);
    for (int z = 0; z < Ec; z++)
        for (int y = 0; y < Ec; y++)
            for (int x = 0; x < Ec; x++) {
                long s = site_index(Ec, x, y, z);
                pts[3 * s] = (double)x * zm; pts[3 * s + 1] = (double)y * zm; pts[3 * s + 2] = (double)z * zm;
            }
    orc_field(kvec, amp, omega, phi, M, xc, pts, n3, t, val);
    for (int c = 0; c < 3; c++)
        for (long s = 0; s < n3; s++) out[c * n3 + s] = val[3 * s + c];
    free(pts);
    free(val);
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
