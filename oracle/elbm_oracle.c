/*
 * FP64 CPU oracle for the two-population compressible lattice Boltzmann model of
 * Saadat, Hosseini, Dorschner & Karlin, "Extended Lattice Boltzmann Model for Gas
 * Dynamics" (arXiv:2102.09512).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * statement of the method that the CUDA path is checked against.  Only the tests,
 * the smoke check and the bench's CPU-baseline leg may load it; the product path
 * never does.  It shares no code, header, table or helper with the CUDA library.
 *
 * Everything is FP64, node-major (array-of-structures: f[node*Q + i]), one node
 * at a time, in the order of one time step:
 *   1. moments rho, u, T at every node                      (Eqs. density, momentum,
 *                                                             energy, U, E)
 *   2. anomaly Q~_aaa at every node                          (Eq. anomalya)
 *   3. its derivative, first-order upwind or central         (Sec. III.A)
 *   4. collision of both populations at every node           (Eqs. fLBGK, gLBGK)
 *   5./6. pull streaming, ghost values by index mapping      (left-hand sides of
 *                                                             Eqs. fLBGK, gLBGK)
 *
 * The g-equilibrium is evaluated from its operator definition (Eq. geq_i): the
 * product of the Psi triplets with xi_a -> O_a and P_aa -> O_a^2 is expanded into
 * monomials O_x^l O_y^m O_z^n (l,m,n <= 2), each applied to the generating
 * function E = Cv T + u^2/2 held as a polynomial in (u_x,u_y,u_z) (Eq. Operator).
 *
 * Readings where the paper is silent:
 *  - the upwind sign is the sign of u_a at the node where the derivative is taken,
 *    strict '>' (a tie takes the forward difference);
 *  - Q~ is taken at the same time level as the collision (post-stream moments);
 *  - P in q* is the full pressure tensor of the pre-collision populations and
 *    P^eq is the non-extended rho T I + rho u u;
 *  - div Q~ in q* is diag(D_x, D_y, D_z), the same discrete derivative as in P^ex;
 *  - omega and omega_1 are node-local, from the local pressure P = rho T;
 *  - boundaries: a periodic axis wraps indices; a zero-gradient face copies the
 *    adjacent interior node (its post-collision populations and its Q~) into the
 *    ghost, i.e. the index is clamped; a fixed-state face (a supersonic inflow)
 *    holds in its ghost the equilibrium populations f^eq, g^eq of a prescribed
 *    uniform state, which is also their post-collision value (a uniform
 *    equilibrium state has no gradients and no non-equilibrium part), and that
 *    state's Q~; a ghost beyond a fixed face on any axis is a fixed ghost;
 *  - D2Q9 is the same product form over x and y, with Cv = 1/(gamma-1);
 *  - the caloric equation of state is either constant Cv = 1/(gamma-1) or a cubic
 *    Cv(T); U(T) enters g^eq as the constant term of the generating function and T is
 *    recovered from U by Newton's method.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int D;                 /* 2 (D2Q9) or 3 (D3Q27)                                 */
    int nx, ny, nz;        /* nz = 1 when D = 2                                      */
    double gamma;          /* adiabatic exponent, Cv = R/(gamma-1), R = 1            */
    double Pr;             /* Prandtl number, Eq. Pr                                 */
    double mu0, T0, mu_exp;/* mu = mu0 (T/T0)^mu_exp (mu_exp = 0: constant mu)       */
    int bc[6];             /* faces -x,+x,-y,+y,-z,+z: 0 periodic, 1 zero-gradient,
                              2 fixed state (supersonic inflow)                      */
    int deriv;             /* 0 first-order upwind, 1 second-order central           */
    int correction;        /* 1 extended equilibrium (the method); 0 plain f^eq      */
    double fix_rho, fix_u[3], fix_T;   /* the state of every fixed-state face        */
    int eos;               /* 0: constant Cv = 1/(gamma-1); 1: Cv(T) = cv[0] + cv[1] T
                              + cv[2] T^2 + cv[3] T^3 (a general caloric ideal gas)   */
    double cv[4];
} orc_params;

/* ----------------------------------------------------------------------------
 * Lattice.  Q = 3^D; direction i has components c_a = ((i / 3^a) mod 3) - 1.
 * (Eq. d3q27vel; D2Q9 is its two-dimensional analogue.)
 * -------------------------------------------------------------------------- */
static int orc_Q(const orc_params *p) { return p->D == 3 ? 27 : 9; }

static void orc_c(int i, int D, int c[3]) {
    c[0] = (i % 3) - 1;
    c[1] = ((i / 3) % 3) - 1;
    c[2] = D == 3 ? ((i / 9) % 3) - 1 : 0;
}

int orc_velocity(int D, int i, int *c3) { orc_c(i, D, c3); return 0; }

/* ----------------------------------------------------------------------------
 * Psi triplet (Eqs. phi0S, phiPlusS, phiMinusS) and the product form
 * (Eq. productform).
 * -------------------------------------------------------------------------- */
static double psi(int c, double xi, double P) {
    if (c == 0) return 1.0 - P;
    if (c == 1) return 0.5 * (xi + P);
    return 0.5 * (-xi + P);
}

static double product_form(const int c[3], int D, const double xi[3], const double P[3]) {
    double v = 1.0;
    for (int a = 0; a < D; ++a) v *= psi(c[a], xi[a], P[a]);
    return v;
}

/* f^eq (Eq. 27eq) with P_aa = T + u_a^2 (Eqs. ci_f, Pi_f), and the extended
 * equilibrium f^ex (Eq. extf) with P_aa^ex = P_aa^eq + dt (2-w)/(2 rho w) d_a Q~_aaa
 * (Eq. Pa_star, dt = 1).  dQ may be NULL for f^eq. */
void orc_fex(const orc_params *p, double rho, const double u[3], double T,
             double omega, const double dQ[3], double *f_out) {
    const int Q = orc_Q(p), D = p->D;
    double P[3] = {0, 0, 0}, xi[3] = {0, 0, 0};
    for (int a = 0; a < D; ++a) {
        xi[a] = u[a];
        P[a] = T + u[a] * u[a];
        if (dQ) P[a] += (2.0 - omega) / (2.0 * rho * omega) * dQ[a];
    }
    for (int i = 0; i < Q; ++i) {
        int c[3];
        orc_c(i, D, c);
        f_out[i] = rho * product_form(c, D, xi, P);
    }
}

/* ----------------------------------------------------------------------------
 * Polynomials in (u_x, u_y, u_z) of degree <= 4 in each variable; the operator
 * O_a A = T dA/du_a + u_a A (Eq. Operator, R = 1) acts on them.
 * -------------------------------------------------------------------------- */
#define PDEG 5
typedef struct { double c[PDEG][PDEG][PDEG]; } poly3;

static void poly_apply_O(poly3 *out, const poly3 *in, int axis, double T) {
    memset(out, 0, sizeof(*out));
    for (int a = 0; a < PDEG; ++a)
        for (int b = 0; b < PDEG; ++b)
            for (int k = 0; k < PDEG; ++k) {
                double v = in->c[a][b][k];
                if (v == 0.0) continue;
                int e[3] = {a, b, k};
                /* T d/du_axis */
                if (e[axis] > 0) {
                    int d[3] = {a, b, k};
                    d[axis] -= 1;
                    out->c[d[0]][d[1]][d[2]] += T * (double)e[axis] * v;
                }
                /* u_axis * (.) ; the degree stays <= 4 because at most two
                 * operators act per axis on the quadratic generating function */
                int m[3] = {a, b, k};
                m[axis] += 1;
                if (m[axis] < PDEG) out->c[m[0]][m[1]][m[2]] += v;
                else abort();
            }
}

static double poly_eval(const poly3 *p, const double u[3]) {
    double s = 0.0;
    for (int a = 0; a < PDEG; ++a)
        for (int b = 0; b < PDEG; ++b)
            for (int k = 0; k < PDEG; ++k) {
                double v = p->c[a][b][k];
                if (v == 0.0) continue;
                s += v * pow(u[0], a) * pow(u[1], b) * pow(u[2], k);
            }
    return s;
}

/* Caloric equation of state (Eq. U, reference temperature 0, R = 1): the specific
 * heat Cv(T), the internal energy U(T) = int_0^T Cv dT, and its inverse. */
static double Cv_of_T(const orc_params *p, double T) {
    if (p->eos == 0) return 1.0 / (p->gamma - 1.0);
    return p->cv[0] + T * (p->cv[1] + T * (p->cv[2] + T * p->cv[3]));
}

static double U_of_T(const orc_params *p, double T) {
    if (p->eos == 0) return T / (p->gamma - 1.0);
    return T * (p->cv[0] + T * (p->cv[1] / 2.0 + T * (p->cv[2] / 3.0 + T * p->cv[3] / 4.0)));
}

/* T with U(T) = U: Newton's method on the monotone U (Cv > 0), from the estimate with
 * Cv(0), to a relative step of 1e-15. */
static double T_of_U(const orc_params *p, double U) {
    if (p->eos == 0) return U * (p->gamma - 1.0);
    double T = U / p->cv[0];
    for (int k = 0; k < 100; ++k) {
        const double dT = (U_of_T(p, T) - U) / Cv_of_T(p, T);
        T -= dT;
        if (fabs(dT) <= 1e-15 * fabs(T)) break;
    }
    return T;
}

/* Generating function E = U(T) + u^2/2 (Eqs. U, E); the operators act on u only, so
 * U(T) enters as the constant term. */
static void energy_poly(const orc_params *p, double T, poly3 *E) {
    memset(E, 0, sizeof(*E));
    E->c[0][0][0] = U_of_T(p, T);
    E->c[2][0][0] = 0.5;
    E->c[0][2][0] = 0.5;
    if (p->D == 3) E->c[0][0][2] = 0.5;
}

/* G_lmn = rho O_x^l O_y^m O_z^n E for l,m,n in {0,1,2} (Eq. Ecompact);
 * G[l][m][n], n = 0 only in 2D. */
void orc_energy_moments(const orc_params *p, double rho, const double u[3], double T,
                        double G[3][3][3]) {
    poly3 E, Ax[3], Axy[3][3], tmp;
    energy_poly(p, T, &E);
    Ax[0] = E;
    poly_apply_O(&Ax[1], &Ax[0], 0, T);
    poly_apply_O(&Ax[2], &Ax[1], 0, T);
    double uu[3] = {u[0], u[1], p->D == 3 ? u[2] : 0.0};
    for (int l = 0; l < 3; ++l) {
        Axy[l][0] = Ax[l];
        poly_apply_O(&Axy[l][1], &Axy[l][0], 1, T);
        poly_apply_O(&Axy[l][2], &Axy[l][1], 1, T);
        for (int m = 0; m < 3; ++m) {
            if (p->D == 2) {
                G[l][m][0] = rho * poly_eval(&Axy[l][m], uu);
                G[l][m][1] = G[l][m][2] = 0.0;
                continue;
            }
            poly3 cur = Axy[l][m];
            for (int n = 0; n < 3; ++n) {
                G[l][m][n] = rho * poly_eval(&cur, uu);
                if (n < 2) { poly_apply_O(&tmp, &cur, 2, T); cur = tmp; }
            }
        }
    }
}

/* Coefficient of O^k in Psi_c(O, O^2): Psi_0 = 1 - O^2, Psi_{+-1} = (+-O + O^2)/2. */
static double psi_op_coeff(int c, int k) {
    if (c == 0) return k == 0 ? 1.0 : (k == 2 ? -1.0 : 0.0);
    if (k == 0) return 0.0;
    if (k == 1) return 0.5 * (double)c;
    return 0.5;
}

/* g^eq_i = rho Psi_cx(O_x,O_x^2) Psi_cy(O_y,O_y^2) Psi_cz(O_z,O_z^2) E (Eq. geq_i). */
void orc_geq(const orc_params *p, double rho, const double u[3], double T, double *g_out) {
    double G[3][3][3];
    orc_energy_moments(p, rho, u, T, G);
    const int Q = orc_Q(p), D = p->D;
    for (int i = 0; i < Q; ++i) {
        int c[3];
        orc_c(i, D, c);
        double s = 0.0;
        for (int l = 0; l < 3; ++l)
            for (int m = 0; m < 3; ++m)
                for (int n = 0; n < (D == 3 ? 3 : 1); ++n) {
                    double coef = psi_op_coeff(c[0], l) * psi_op_coeff(c[1], m);
                    if (D == 3) coef *= psi_op_coeff(c[2], n);
                    s += coef * G[l][m][n];
                }
        g_out[i] = s;
    }
}

/* ----------------------------------------------------------------------------
 * Moments (Eqs. density, momentum, energy, P) and temperature from E (Eq. E).
 * -------------------------------------------------------------------------- */
typedef struct {
    double rho, u[3], E, T, P[3][3];
} orc_moments;

static void node_moments(const orc_params *p, const double *f, const double *g, orc_moments *m) {
    const int Q = orc_Q(p), D = p->D;
    double rho = 0, j[3] = {0, 0, 0}, rE = 0, P[3][3] = {{0}};
    for (int i = 0; i < Q; ++i) {
        int c[3];
        orc_c(i, D, c);
        rho += f[i];
        rE += g[i];
        for (int a = 0; a < 3; ++a) {
            j[a] += c[a] * f[i];
            for (int b = 0; b < 3; ++b) P[a][b] += c[a] * c[b] * f[i];
        }
    }
    m->rho = rho;
    double u2 = 0;
    for (int a = 0; a < 3; ++a) { m->u[a] = j[a] / rho; u2 += m->u[a] * m->u[a]; }
    m->E = rE / rho;
    m->T = T_of_U(p, m->E - 0.5 * u2);
    memcpy(m->P, P, sizeof(P));
}

/* Anomaly Q~_aaa = rho u_a (1 - 3 T) - rho u_a^3 (Eq. anomalya, R = 1). */
static double anomaly(double rho, double ua, double T) {
    return rho * ua * (1.0 - 3.0 * T) - rho * ua * ua * ua;
}

/* omega from mu = (1/omega - 1/2) P dt (Eq. mu), omega_1 from
 * Pr = omega_1 (2 - omega) / (omega (2 - omega_1)) (Eq. Pr). */
void orc_rates(const orc_params *p, double rho, double T, double *omega, double *omega1) {
    double mu = p->mu0;
    if (p->mu_exp != 0.0) mu = p->mu0 * pow(T / p->T0, p->mu_exp);
    const double P = rho * T;
    const double w = 1.0 / (mu / P + 0.5);
    *omega = w;
    *omega1 = 2.0 * p->Pr * w / (2.0 - w + p->Pr * w);
}

/* One collision (Eqs. fLBGK, gLBGK) at one node, given its pre-collision
 * populations and the discrete derivative dQ_a of Q~_aaa at that node.
 * Also returns f^ex, g^eq, g* when the pointers are non-NULL. */
void orc_collide_node(const orc_params *p, const double *f, const double *g, const double dQ[3],
                      double *f_post, double *g_post,
                      double *fex_out, double *geq_out, double *gstar_out) {
    const int Q = orc_Q(p), D = p->D;
    orc_moments m;
    node_moments(p, f, g, &m);
    double omega, omega1;
    orc_rates(p, m.rho, m.T, &omega, &omega1);

    double fex[27], geq[27], gst[27];
    orc_fex(p, m.rho, m.u, m.T, omega, p->correction ? dQ : NULL, fex);
    orc_geq(p, m.rho, m.u, m.T, geq);

    /* q^eq = rho O_a E (Eq. qeq), first-order energy moments */
    double G[3][3][3];
    orc_energy_moments(p, m.rho, m.u, m.T, G);
    double qeq[3] = {G[1][0][0], G[0][1][0], D == 3 ? G[0][0][1] : 0.0};

    /* q* = q^eq + u . (P - P^eq + dt/2 div Q~)  (Eq. qstar1), P^eq = rho T I + rho u u
     * (Eqs. Peq, PMB), div Q~ = diag(dQ). */
    double qstar[3];
    for (int a = 0; a < D; ++a) {
        double s = 0.0;
        for (int b = 0; b < D; ++b) {
            double Peq = m.rho * m.u[a] * m.u[b] + (a == b ? m.rho * m.T : 0.0);
            double divQ = (a == b && p->correction) ? dQ[a] : 0.0;
            s += m.u[b] * (m.P[b][a] - Peq + 0.5 * divQ);
        }
        qstar[a] = qeq[a] + s;
    }
    if (D == 2) qstar[2] = 0.0;

    /* g* (Eq. gstar): only the |c_i|^2 = 1 populations carry the flux change */
    for (int i = 0; i < Q; ++i) {
        int c[3];
        orc_c(i, D, c);
        int c2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
        gst[i] = geq[i];
        if (c2 == 1)
            for (int a = 0; a < D; ++a) gst[i] += 0.5 * c[a] * (qstar[a] - qeq[a]);
    }

    for (int i = 0; i < Q; ++i) {
        f_post[i] = f[i] + omega * (fex[i] - f[i]);
        g_post[i] = g[i] + omega1 * (geq[i] - g[i]) + (omega - omega1) * (geq[i] - gst[i]);
        if (fex_out) fex_out[i] = fex[i];
        if (geq_out) geq_out[i] = geq[i];
        if (gstar_out) gstar_out[i] = gst[i];
    }
}

/* ----------------------------------------------------------------------------
 * Grid indexing.  A periodic axis wraps, a zero-gradient axis clamps (the ghost
 * holds a copy of the adjacent interior node).
 * -------------------------------------------------------------------------- */
static int map_axis(int x, int n, int bc_lo, int bc_hi) {
    if (x < 0) return bc_lo == 0 ? ((x % n) + n) % n : 0;
    if (x >= n) return bc_hi == 0 ? x % n : n - 1;
    return x;
}

/* Node index of (x,y,z) after the boundary maps, or -1 for a ghost beyond a
 * fixed-state face. */
static long node_of(const orc_params *p, int x, int y, int z) {
    const int v[3] = {x, y, z}, n[3] = {p->nx, p->ny, p->nz};
    for (int a = 0; a < 3; ++a)
        if ((v[a] < 0 && p->bc[2 * a] == 2) || (v[a] >= n[a] && p->bc[2 * a + 1] == 2)) return -1;
    x = map_axis(x, p->nx, p->bc[0], p->bc[1]);
    y = map_axis(y, p->ny, p->bc[2], p->bc[3]);
    z = map_axis(z, p->nz, p->bc[4], p->bc[5]);
    return (long)x + (long)p->nx * ((long)y + (long)p->ny * (long)z);
}

static long n_nodes(const orc_params *p) { return (long)p->nx * p->ny * p->nz; }

/* Initial populations: f = f^eq(rho,u,T), g = g^eq(rho,u,T), no non-equilibrium part. */
int orc_init(const orc_params *p, const double *rho, const double *u, const double *T,
             double *f, double *g) {
    const long N = n_nodes(p);
    const int Q = orc_Q(p);
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        double un[3] = {u[n], u[N + n], p->D == 3 ? u[2 * N + n] : 0.0};
        orc_fex(p, rho[n], un, T[n], 1.0, NULL, f + n * Q);
        orc_geq(p, rho[n], un, T[n], g + n * Q);
    }
    return 0;
}

/* rho, u (D x N, component-major) and T from the populations. */
int orc_fields(const orc_params *p, const double *f, const double *g,
               double *rho, double *u, double *T) {
    const long N = n_nodes(p);
    const int Q = orc_Q(p);
#pragma omp parallel for schedule(static)
    for (long n = 0; n < N; ++n) {
        orc_moments m;
        node_moments(p, f + n * Q, g + n * Q, &m);
        rho[n] = m.rho;
        for (int a = 0; a < p->D; ++a) u[a * N + n] = m.u[a];
        T[n] = m.T;
    }
    return 0;
}

/* Discrete derivative of Q~_aaa along axis a at node (x,y,z) (Sec. III.A):
 * upwind: Q~_{i+1/2} - Q~_{i-1/2} with the interface value taken from the
 * upwind side of u_a at the node; central: (Q~_{i+1} - Q~_{i-1}) / 2. */
static double dQ_axis(const orc_params *p, const double *Qt, const double *uvel,
                      int x, int y, int z, int a) {
    const long N = n_nodes(p);
    int e[3] = {0, 0, 0};
    e[a] = 1;
    long n0 = node_of(p, x, y, z);
    long np = node_of(p, x + e[0], y + e[1], z + e[2]);
    long nm = node_of(p, x - e[0], y - e[1], z - e[2]);
    const double *q = Qt + a * N;
    const double qfix = anomaly(p->fix_rho, p->fix_u[a], p->fix_T);   /* fixed ghost */
    const double q0 = q[n0], qp = np < 0 ? qfix : q[np], qm = nm < 0 ? qfix : q[nm];
    if (p->deriv == 1) return 0.5 * (qp - qm);
    double right = uvel[a * N + n0] > 0.0 ? q0 : qp;   /* Q~ at i+1/2 */
    double left = uvel[a * N + n0] > 0.0 ? qm : q0;    /* Q~ at i-1/2 */
    return right - left;
}

/* nsteps time steps in place (the post-collision copies are allocated here). */
int orc_step(const orc_params *p, double *f, double *g, int nsteps) {
    const long N = n_nodes(p);
    const int Q = orc_Q(p), D = p->D;
    double *fpc = (double *)malloc(sizeof(double) * N * Q);
    double *gpc = (double *)malloc(sizeof(double) * N * Q);
    double *Qt = (double *)malloc(sizeof(double) * 3 * N);
    double *uvel = (double *)malloc(sizeof(double) * 3 * N);
    if (!fpc || !gpc || !Qt || !uvel) { free(fpc); free(gpc); free(Qt); free(uvel); return -1; }
    double ffix[27], gfix[27];   /* ghost populations of a fixed-state face */
    orc_fex(p, p->fix_rho, p->fix_u, p->fix_T, 1.0, NULL, ffix);
    orc_geq(p, p->fix_rho, p->fix_u, p->fix_T, gfix);

    for (int s = 0; s < nsteps; ++s) {
        /* 1-2: moments and anomaly at every node */
#pragma omp parallel for schedule(static)
        for (long n = 0; n < N; ++n) {
            orc_moments m;
            node_moments(p, f + n * Q, g + n * Q, &m);
            for (int a = 0; a < 3; ++a) {
                uvel[a * N + n] = m.u[a];
                Qt[a * N + n] = a < D ? anomaly(m.rho, m.u[a], m.T) : 0.0;
            }
        }
        /* 3-4: derivative and collision at every node */
#pragma omp parallel for schedule(static)
        for (long n = 0; n < N; ++n) {
            int x = (int)(n % p->nx), y = (int)((n / p->nx) % p->ny), z = (int)(n / ((long)p->nx * p->ny));
            double dQ[3] = {0, 0, 0};
            for (int a = 0; a < D; ++a) dQ[a] = dQ_axis(p, Qt, uvel, x, y, z, a);
            orc_collide_node(p, f + n * Q, g + n * Q, dQ, fpc + n * Q, gpc + n * Q, NULL, NULL, NULL);
        }
        /* 5-6: pull streaming f_i(x) <- f_i^pc(x - c_i), ghosts by index mapping;
         * fixed ghosts hold the equilibria of the fixed state */
#pragma omp parallel for schedule(static)
        for (long n = 0; n < N; ++n) {
            int x = (int)(n % p->nx), y = (int)((n / p->nx) % p->ny), z = (int)(n / ((long)p->nx * p->ny));
            for (int i = 0; i < Q; ++i) {
                int c[3];
                orc_c(i, D, c);
                long src = node_of(p, x - c[0], y - c[1], z - c[2]);
                f[n * Q + i] = src < 0 ? ffix[i] : fpc[src * Q + i];
                g[n * Q + i] = src < 0 ? gfix[i] : gpc[src * Q + i];
            }
        }
    }
    free(fpc); free(gpc); free(Qt); free(uvel);
    return 0;
}

/* Totals sum rho, sum rho u_a, sum rho E over all nodes, Neumaier-compensated,
 * in node order (Eqs. density, momentum, energy).  out[5] = {M, Jx, Jy, Jz, E}. */
int orc_conservation(const orc_params *p, const double *f, const double *g, double *out) {
    const long N = n_nodes(p);
    const int Q = orc_Q(p), D = p->D;
    double s[5] = {0}, comp[5] = {0};
    for (long n = 0; n < N; ++n) {
        double v[5] = {0, 0, 0, 0, 0};
        for (int i = 0; i < Q; ++i) {
            int c[3];
            orc_c(i, D, c);
            v[0] += f[n * Q + i];
            v[1] += c[0] * f[n * Q + i];
            v[2] += c[1] * f[n * Q + i];
            v[3] += c[2] * f[n * Q + i];
            v[4] += g[n * Q + i];
        }
        for (int k = 0; k < 5; ++k) {
            double t = s[k] + v[k];
            if (fabs(s[k]) >= fabs(v[k])) comp[k] += (s[k] - t) + v[k];
            else comp[k] += (v[k] - t) + s[k];
            s[k] = t;
        }
    }
    for (int k = 0; k < 5; ++k) out[k] = s[k] + comp[k];
    return 0;
}

int orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
