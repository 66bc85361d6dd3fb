/*
 * FP64 CPU oracle for the lattice Boltzmann scheme with relative velocities
 * (F. Dubois, T. Fevrier, B. Graille, "Lattice Boltzmann schemes with relative
 * velocities", arXiv:1312.3297), D2Q9 lattice with the orthogonal moment set of
 * Section 1.3.
 *
 * TEST INFRASTRUCTURE. This is the plain, slow reference that the GPU library is
 * checked against. Only the test-suite, the smoke check and the benchmark's CPU
 * baseline leg load it. It shares no code, header, table or helper with the CUDA
 * library, and it never calls it.
 *
 * Three steppers, written independently of one another:
 *   definition: Section 1.2 taken literally. Per node the shifted moment matrix
 *               M(u~)_kj = P_k(v_j - u~) is built from the polynomials of
 *               relation (mom), m = M(u~) f, m_eq = M(u~) f_eq, the diagonal
 *               relaxation (relaxationu), and f* = M(u~)^{-1} m* solved by LU with
 *               partial pivoting. Then the exact transport (transport).
 *   shifted:    Section 1.3: fixed moments m(0) = M(0) f, the shifting matrix
 *               T(u~) of relation (matTu) with the blocks of Appendix A, relaxation
 *               of T(u~) m(0) towards T(u~) m_eq(0), and the way back
 *               f* = M(0)^{-1} T(-u~) m*, which is valid by the morphism property
 *               (Proposition "Morphism of groups", Section 1.3). The D_2 block is
 *               the one recomputed from T = M(u~) M(0)^{-1}:
 *               -9/lambda^4 u~^alpha (lambda^2 + 2|u~|^2); the printed block carries
 *               an extra factor 1/2.
 *   mrt:        Section 1.1: d'Humieres fixed-moment MRT with the integer matrix
 *               of relation (matort) and M(0)^{-1} = M(0)^T diag(1/|row_k|^2)
 *               (rows are orthogonal).
 *
 * Readings where the paper is silent (each stated where it is used):
 *   - the equilibrium is the second-order polynomial D2Q9 equilibrium
 *     f_eq,j = w_j rho (1 + 3 v.u/l^2 + 9/2 (v.u)^2/l^4 - 3/2 |u|^2/l^2),
 *     u = q/rho, w = (4/9, 1/9 x4, 1/36 x4); the paper allows any equilibrium
 *     independent of u~ (Section 1.2);
 *   - lattice units dx = 1, so dt = 1/lambda (relation (lambda)) and v_j dt is one
 *     lattice link;
 *   - the relative velocity is u~ = 0, u~ = q/rho (from the moments of the state
 *     being relaxed; q and rho are collision invariants), or a prescribed field
 *     u~(x,t) = A u~0(x) cos(2 pi t / P) evaluated at the time index t of the
 *     collision; u~0 is a caller field or the analytic (cos 2pi y/Ly, sin 2pi x/Lx).
 *
 * Layout: structure of arrays, f[(j*ny + y)*nx + x], x fastest; periodic lattice.
 * Build with -ffp-contract=off: the ũ = 0 bit-for-bit check relies on no fused
 * multiply-adds being introduced.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define Q 9

/* Velocity set of Section 1.3 in the paper's order, in units of lambda. */
static const int CX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

int orc_q(void) { return Q; }

/* The D2Q9 velocities v_j = lambda * (CX[j], CY[j]) (Section 1.3). */
void orc_velocities(double lambda, double* vx, double* vy) {
    for (int j = 0; j < Q; ++j) {
        vx[j] = lambda * CX[j];
        vy[j] = lambda * CY[j];
    }
}

/* Polynomial P_k(X, Y) of the orthogonal moment set, relation (mom). */
double orc_poly(int k, double X, double Y, double l) {
    double r2 = X * X + Y * Y;
    switch (k) {
        case 0: return 1.0;
        case 1: return X;
        case 2: return Y;
        case 3: return (3.0 * r2 - 4.0 * l * l) / (l * l);
        case 4: return (X * X - Y * Y) / (l * l);
        case 5: return X * Y / (l * l);
        case 6: return X * (3.0 * r2 - 5.0 * l * l) / (l * l * l);
        case 7: return Y * (3.0 * r2 - 5.0 * l * l) / (l * l * l);
        case 8: return (4.5 * r2 * r2 - 10.5 * l * l * r2 + 4.0 * l * l * l * l) / (l * l * l * l);
        default: return NAN;
    }
}

/* Shifted moment matrix M(u~)_kj = P_k(v_j - u~), relation (MatMu); row-major M[k*9+j]. */
void orc_moment_matrix(double ux, double uy, double l, double* M) {
    for (int k = 0; k < Q; ++k)
        for (int j = 0; j < Q; ++j)
            M[k * Q + j] = orc_poly(k, l * CX[j] - ux, l * CY[j] - uy, l);
}

/* Second-order polynomial equilibrium (reading: the paper leaves f_eq general). */
void orc_feq(double rho, double ux, double uy, double l, double* feq) {
    static const double W[Q] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                                1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
    double l2 = l * l;
    double uu = ux * ux + uy * uy;
    for (int j = 0; j < Q; ++j) {
        double vu = l * CX[j] * ux + l * CY[j] * uy;
        feq[j] = W[j] * rho * (1.0 + 3.0 * vu / l2 + 4.5 * vu * vu / (l2 * l2) - 1.5 * uu / l2);
    }
}

/* Conserved moments of relation (rhoq): rho = sum f_j, q = sum v_j f_j. */
static void conserved(const double* f, double l, double* rho, double* qx, double* qy) {
    double r = 0.0, a = 0.0, b = 0.0;
    for (int j = 0; j < Q; ++j) {
        r += f[j];
        a += l * CX[j] * f[j];
        b += l * CY[j] * f[j];
    }
    *rho = r;
    *qx = a;
    *qy = b;
}

/* Solve A x = b (n = 9) by Gaussian elimination with partial pivoting.
 * A and b are overwritten. Returns 0, or -1 if a pivot is exactly zero. */
int orc_lu_solve(double* A, double* b, double* x) {
    for (int c = 0; c < Q; ++c) {
        int p = c;
        double best = fabs(A[c * Q + c]);
        for (int r = c + 1; r < Q; ++r) {
            double v = fabs(A[r * Q + c]);
            if (v > best) { best = v; p = r; }
        }
        if (best == 0.0) return -1;
        if (p != c) {
            for (int k = 0; k < Q; ++k) {
                double t = A[c * Q + k]; A[c * Q + k] = A[p * Q + k]; A[p * Q + k] = t;
            }
            double t = b[c]; b[c] = b[p]; b[p] = t;
        }
        for (int r = c + 1; r < Q; ++r) {
            double m = A[r * Q + c] / A[c * Q + c];
            for (int k = c; k < Q; ++k) A[r * Q + k] -= m * A[c * Q + k];
            b[r] -= m * b[c];
        }
    }
    for (int r = Q - 1; r >= 0; --r) {
        double acc = b[r];
        for (int k = r + 1; k < Q; ++k) acc -= A[r * Q + k] * x[k];
        x[r] = acc / A[r * Q + r];
    }
    return 0;
}

/* One relaxation at a node, Section 1.2 as defined: m = M(u~) f (ftomu),
 * m_eq = M(u~) f_eq, m*_k = m_k + s_k (m_eq,k - m_k) (relaxationu),
 * f* = M(u~)^{-1} m*. Returns 0 or -1 (singular matrix, never for D2Q9). */
int orc_collide_definition(const double* f, double utx, double uty, double l,
                           const double* s, double* fstar) {
    double M[Q * Q], feq[Q], m[Q], meq[Q], ms[Q];
    double rho, qx, qy;
    conserved(f, l, &rho, &qx, &qy);
    orc_feq(rho, qx / rho, qy / rho, l, feq);
    orc_moment_matrix(utx, uty, l, M);
    for (int k = 0; k < Q; ++k) {
        double a = 0.0, b = 0.0;
        for (int j = 0; j < Q; ++j) {
            a += M[k * Q + j] * f[j];
            b += M[k * Q + j] * feq[j];
        }
        m[k] = a;
        meq[k] = b;
    }
    for (int k = 0; k < Q; ++k) {
        ms[k] = m[k] + s[k] * (meq[k] - m[k]);
    }
    return orc_lu_solve(M, ms, fstar);
}

/* Shifting matrix T(u~) of relation (matTu), blocks of Appendix A; row-major.
 * Column/row order: rho, q_x, q_y, e, p_xx, p_xy, q_x(3rd), q_y(3rd), eps. */
void orc_shift_matrix(double ux, double uy, double l, double* T) {
    double l2 = l * l, l3 = l2 * l, l4 = l2 * l2;
    double uu = ux * ux + uy * uy;
    memset(T, 0, sizeof(double) * Q * Q);
    for (int k = 0; k < Q; ++k) T[k * Q + k] = 1.0;
    /* A */
    T[1 * Q + 0] = -ux;
    T[2 * Q + 0] = -uy;
    /* B1 */
    T[3 * Q + 0] = 3.0 * uu / l2;
    T[4 * Q + 0] = (ux * ux - uy * uy) / l2;
    T[5 * Q + 0] = ux * uy / l2;
    /* B2 */
    T[3 * Q + 1] = -6.0 * ux / l2;  T[3 * Q + 2] = -6.0 * uy / l2;
    T[4 * Q + 1] = -2.0 * ux / l2;  T[4 * Q + 2] = 2.0 * uy / l2;
    T[5 * Q + 1] = -uy / l2;        T[5 * Q + 2] = -ux / l2;
    /* C1 */
    T[6 * Q + 0] = -3.0 * ux * (uu + l2) / l3;
    T[7 * Q + 0] = -3.0 * uy * (uu + l2) / l3;
    /* C2 */
    T[6 * Q + 1] = 3.0 * (uu + 2.0 * ux * ux) / l3;  T[6 * Q + 2] = 6.0 * ux * uy / l3;
    T[7 * Q + 1] = 6.0 * ux * uy / l3;               T[7 * Q + 2] = 3.0 * (uu + 2.0 * uy * uy) / l3;
    /* C3 */
    T[6 * Q + 3] = -2.0 * ux / l;  T[6 * Q + 4] = -3.0 * ux / l;
    T[6 * Q + 5] = -6.0 * uy / l;
    T[7 * Q + 3] = -2.0 * uy / l;  T[7 * Q + 4] = 3.0 * uy / l;   T[7 * Q + 5] = -6.0 * ux / l;
    /* D1 */
    T[8 * Q + 0] = 4.5 * (uu * uu + 3.0 * l2 * uu) / l4;
    /* D2, recomputed from T = M(u~) M(0)^{-1} (the printed block has an extra 1/2) */
    T[8 * Q + 1] = -9.0 * ux * (l2 + 2.0 * uu) / l4;
    T[8 * Q + 2] = -9.0 * uy * (l2 + 2.0 * uu) / l4;
    /* D3 */
    T[8 * Q + 3] = 6.0 * uu / l2;
    T[8 * Q + 4] = 9.0 * (ux * ux - uy * uy) / l2;
    T[8 * Q + 5] = 36.0 * ux * uy / l2;
    /* D4 */
    T[8 * Q + 6] = -6.0 * ux / l;
    T[8 * Q + 7] = -6.0 * uy / l;
}

/* M(0) built from the polynomials and its squared row norms (rows are orthogonal). */
static void fixed_matrix(double l, double* M0, double* norm2) {
    orc_moment_matrix(0.0, 0.0, l, M0);
    for (int k = 0; k < Q; ++k) {
        double a = 0.0;
        for (int j = 0; j < Q; ++j) a += M0[k * Q + j] * M0[k * Q + j];
        norm2[k] = a;
    }
}

/* One relaxation at a node in the shifted form of Section 1.3 (see file header). */
void orc_collide_shifted(const double* f, double utx, double uty, double l,
                         const double* s, double* fstar) {
    double M0[Q * Q], n2[Q], T[Q * Q], Tm[Q * Q], feq[Q];
    double m0[Q], meq0[Q], m[Q], meq[Q], ms[Q], mb[Q];
    double rho, qx, qy;
    fixed_matrix(l, M0, n2);
    conserved(f, l, &rho, &qx, &qy);
    orc_feq(rho, qx / rho, qy / rho, l, feq);
    for (int k = 0; k < Q; ++k) {
        double a = 0.0, b = 0.0;
        for (int j = 0; j < Q; ++j) {
            a += M0[k * Q + j] * f[j];
            b += M0[k * Q + j] * feq[j];
        }
        m0[k] = a;
        meq0[k] = b;
    }
    orc_shift_matrix(utx, uty, l, T);
    orc_shift_matrix(-utx, -uty, l, Tm);
    for (int k = 0; k < Q; ++k) {
        double a = 0.0, b = 0.0;
        for (int c = 0; c < Q; ++c) {
            a += T[k * Q + c] * m0[c];
            b += T[k * Q + c] * meq0[c];
        }
        m[k] = a;
        meq[k] = b;
    }
    for (int k = 0; k < Q; ++k) ms[k] = m[k] + s[k] * (meq[k] - m[k]);
    for (int k = 0; k < Q; ++k) {
        double a = 0.0;
        for (int c = 0; c < Q; ++c) a += Tm[k * Q + c] * ms[c];
        mb[k] = a;
    }
    for (int j = 0; j < Q; ++j) {
        double a = 0.0;
        for (int k = 0; k < Q; ++k) a += M0[k * Q + j] * mb[k] / n2[k];
        fstar[j] = a;
    }
}

/* d'Humieres fixed-moment MRT relaxation at a node (Section 1.1), coded on its own:
 * the integer matrix of relation (matort) is typed in, rows 1 and 2 scaled by lambda. */
void orc_collide_mrt(const double* f, double l, const double* s, double* fstar) {
    static const int MI[Q][Q] = {
        { 1,  1,  1,  1,  1,  1,  1,  1,  1},
        { 0,  1,  0, -1,  0,  1, -1, -1,  1},
        { 0,  0,  1,  0, -1,  1,  1, -1, -1},
        {-4, -1, -1, -1, -1,  2,  2,  2,  2},
        { 0,  1, -1,  1, -1,  0,  0,  0,  0},
        { 0,  0,  0,  0,  0,  1, -1,  1, -1},
        { 0, -2,  0,  2,  0,  1, -1, -1,  1},
        { 0,  0, -2,  0,  2,  1,  1, -1, -1},
        { 4, -2, -2, -2, -2,  1,  1,  1,  1}};
    double M[Q][Q], nrm[Q], feq[Q], m[Q], meq[Q], ms[Q];
    for (int k = 0; k < Q; ++k) {
        double scale = (k == 1 || k == 2) ? l : 1.0;
        double a = 0.0;
        for (int j = 0; j < Q; ++j) {
            M[k][j] = scale * MI[k][j];
            a += M[k][j] * M[k][j];
        }
        nrm[k] = a;
    }
    double rho = 0.0, qx = 0.0, qy = 0.0;
    for (int j = 0; j < Q; ++j) {
        rho += f[j];
        qx += l * CX[j] * f[j];
        qy += l * CY[j] * f[j];
    }
    orc_feq(rho, qx / rho, qy / rho, l, feq);
    for (int k = 0; k < Q; ++k) {
        double a = 0.0, b = 0.0;
        for (int j = 0; j < Q; ++j) {
            a += M[k][j] * f[j];
            b += M[k][j] * feq[j];
        }
        m[k] = a;
        meq[k] = b;
    }
    for (int k = 0; k < Q; ++k) ms[k] = m[k] + s[k] * (meq[k] - m[k]);
    for (int j = 0; j < Q; ++j) {
        double a = 0.0;
        for (int k = 0; k < Q; ++k) a += M[k][j] * ms[k] / nrm[k];
        fstar[j] = a;
    }
}

int orc_collide_geier(const double* f, double utx, double uty, double l, const double* s,
                      double* fstar);
int orc_collide_cascaded(const double* f, double l, const double* s, double* fstar);

/* Relative velocity at node (x, y) and collision time t.
 * mode 0: u~ = 0 (d'Humieres); 1: u~ = q/rho (cascaded-like); 2: prescribed field
 * u~ = amp * u0(x) * cos(2 pi t / period) (no time factor when period <= 0), with
 * u0 = ut0[2][ny][nx] or, when ut0 is NULL, (cos 2 pi y/ny, sin 2 pi x/nx). */
static void relative_velocity(int mode, const double* f, double l, int64_t nx, int64_t ny,
                              int64_t x, int64_t y, const double* ut0, double amp,
                              double period, int64_t t, double* utx, double* uty) {
    if (mode == 0) {
        *utx = 0.0;
        *uty = 0.0;
    } else if (mode == 1) {
        double rho, qx, qy;
        conserved(f, l, &rho, &qx, &qy);
        *utx = qx / rho;
        *uty = qy / rho;
    } else {
        const double twopi = 6.283185307179586476925286766559;
        double tf = period > 0.0 ? cos(twopi * (double)t / period) : 1.0;
        double bx, by;
        if (ut0) {
            bx = ut0[y * nx + x];
            by = ut0[nx * ny + y * nx + x];
        } else {
            bx = cos(twopi * (double)y / (double)ny);
            by = sin(twopi * (double)x / (double)nx);
        }
        *utx = amp * bx * tf;
        *uty = amp * by * tf;
    }
}

/* Relaxation at every node at time t (no transport). method: 0 definition, 1 shifted,
 * 2 mrt (ignores the mode), 3 definition in the Geier basis with the product equilibrium,
 * 4 Geier's cascade of Appendix B (u~ = q/rho, ignores the mode). Returns 0, or -1 on a
 * singular matrix. */
int orc_collide_lattice(int method, int64_t nx, int64_t ny, double l, const double* s,
                        int mode, const double* ut0, double amp, double period, int64_t t,
                        const double* fin, double* fout, int nthreads) {
    int64_t n = nx * ny;
    int status = 0;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(static) num_threads(nthreads) reduction(min : status)
    for (int64_t y = 0; y < ny; ++y) {
        for (int64_t x = 0; x < nx; ++x) {
            double f[Q], fs[Q], utx, uty;
            int64_t i = y * nx + x;
            for (int j = 0; j < Q; ++j) f[j] = fin[j * n + i];
            relative_velocity(mode, f, l, nx, ny, x, y, ut0, amp, period, t, &utx, &uty);
            if (method == 0) {
                if (orc_collide_definition(f, utx, uty, l, s, fs) != 0) status = -1;
            } else if (method == 1) {
                orc_collide_shifted(f, utx, uty, l, s, fs);
            } else if (method == 2) {
                orc_collide_mrt(f, l, s, fs);
            } else if (method == 3) {
                if (orc_collide_geier(f, utx, uty, l, s, fs) != 0) status = -1;
            } else {
                if (orc_collide_cascaded(f, l, s, fs) != 0) status = -1;
            }
            for (int j = 0; j < Q; ++j) fout[j * n + i] = fs[j];
        }
    }
    return status;
}

/* Exact transport, relation (transport): f_j(x, t+dt) = f*_j(x - v_j dt, t), periodic. */
void orc_stream(int64_t nx, int64_t ny, const double* fin, double* fout, int nthreads) {
    int64_t n = nx * ny;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int64_t y = 0; y < ny; ++y) {
        for (int64_t x = 0; x < nx; ++x) {
            for (int j = 0; j < Q; ++j) {
                int64_t xs = ((x - CX[j]) % nx + nx) % nx;
                int64_t ys = ((y - CY[j]) % ny + ny) % ny;
                fout[j * n + y * nx + x] = fin[j * n + ys * nx + xs];
            }
        }
    }
}

/* nsteps time steps (relaxation at times t0 .. t0+nsteps-1, each followed by the
 * transport). f holds the pre-collision state f(t0) on entry and f(t0+nsteps) on
 * exit; work is a caller buffer of the same size. Returns 0 or -1. */
int orc_run(int method, int64_t nx, int64_t ny, double l, const double* s, int mode,
            const double* ut0, double amp, double period, int64_t t0, int64_t nsteps,
            double* f, double* work, int nthreads) {
    for (int64_t k = 0; k < nsteps; ++k) {
        if (orc_collide_lattice(method, nx, ny, l, s, mode, ut0, amp, period, t0 + k, f,
                                work, nthreads) != 0)
            return -1;
        orc_stream(nx, ny, work, f, nthreads);
    }
    return 0;
}

/* f(x, 0) = f_eq(rho(x), u(x)) (reading: the paper does not fix the initial state). */
void orc_init_equilibrium(int64_t nx, int64_t ny, double l, const double* rho,
                          const double* ux, const double* uy, double* f) {
    int64_t n = nx * ny;
    for (int64_t i = 0; i < n; ++i) {
        double feq[Q];
        orc_feq(rho[i], ux[i], uy[i], l, feq);
        for (int j = 0; j < Q; ++j) f[j * n + i] = feq[j];
    }
}

/* Density and velocity u = q/rho at every node, relation (rhoq). */
void orc_moments(int64_t nx, int64_t ny, double l, const double* f, double* rho,
                 double* ux, double* uy) {
    int64_t n = nx * ny;
    for (int64_t i = 0; i < n; ++i) {
        double g[Q], r, a, b;
        for (int j = 0; j < Q; ++j) g[j] = f[j * n + i];
        conserved(g, l, &r, &a, &b);
        rho[i] = r;
        ux[i] = a / r;
        uy[i] = b / r;
    }
}

/* ------------------------------------------------------------------------------------
 * Geier's cascaded scheme as a scheme with relative velocities (proposition of Section
 * 1.3 on the cascaded scheme, Appendix B).
 *
 * Basis (relation (polgeier)): 1, X, Y, X^2+Y^2, X^2-Y^2, XY, XY^2, X^2Y, X^2Y^2, divided by
 * lambda^degree from degree 2 on. Equilibrium (reading: the paper says Geier's equilibria
 * come from the Maxwellian but does not print them): the populations whose moments in this
 * basis, shifted by the fluid velocity u = q/rho, are those of the Maxwellian,
 * (rho, 0, 0, 2 rho c^2, 0, 0, 0, 0, rho c^4) with c^2 = lambda^2/3. On the D2Q9 velocities
 * this is the product form f_eq(v) = rho phi(v_x, u_x) phi(v_y, u_y) with
 * phi(0, a) = 2/3 - a^2/lambda^2, phi(+-lambda, a) = (1/3 + a^2/lambda^2 +- a/lambda)/2.
 */
double orc_poly_geier(int k, double X, double Y, double l) {
    double l2 = l * l, l3 = l2 * l, l4 = l2 * l2;
    switch (k) {
        case 0: return 1.0;
        case 1: return X;
        case 2: return Y;
        case 3: return (X * X + Y * Y) / l2;
        case 4: return (X * X - Y * Y) / l2;
        case 5: return X * Y / l2;
        case 6: return X * Y * Y / l3;
        case 7: return X * X * Y / l3;
        case 8: return X * X * Y * Y / l4;
        default: return NAN;
    }
}

void orc_moment_matrix_geier(double ux, double uy, double l, double* M) {
    for (int k = 0; k < Q; ++k)
        for (int j = 0; j < Q; ++j)
            M[k * Q + j] = orc_poly_geier(k, l * CX[j] - ux, l * CY[j] - uy, l);
}

static double phi1(int c, double a) {
    if (c == 0) return 2.0 / 3.0 - a * a;
    return 0.5 * (1.0 / 3.0 + a * a + c * a);
}

void orc_feq_product(double rho, double ux, double uy, double l, double* feq) {
    for (int j = 0; j < Q; ++j) feq[j] = rho * phi1(CX[j], ux / l) * phi1(CY[j], uy / l);
}

/* Relaxation of Section 1.2 in the Geier basis with the product equilibrium. */
int orc_collide_geier(const double* f, double utx, double uty, double l, const double* s,
                      double* fstar) {
    double M[Q * Q], feq[Q], m[Q], meq[Q], ms[Q];
    double rho, qx, qy;
    conserved(f, l, &rho, &qx, &qy);
    orc_feq_product(rho, qx / rho, qy / rho, l, feq);
    orc_moment_matrix_geier(utx, uty, l, M);
    for (int k = 0; k < Q; ++k) {
        double a = 0.0, b = 0.0;
        for (int j = 0; j < Q; ++j) {
            a += M[k * Q + j] * f[j];
            b += M[k * Q + j] * feq[j];
        }
        m[k] = a;
        meq[k] = b;
    }
    for (int k = 0; k < Q; ++k) {
        ms[k] = m[k] + s[k] * (meq[k] - m[k]);
    }
    return orc_lu_solve(M, ms, fstar);
}

/* Geier's cascaded relaxation written as in Appendix B, coded separately from the above:
 * moments m_g(u) in Geier's original set 1, X, Y, X^2, Y^2, XY, XY^2, X^2Y, X^2Y^2 shifted
 * by u = q/rho; the collision f* = f + M(0)^T g (relation (relgeier), M(0) of relation
 * (matort)) with g from C(u) g = Lambda (m_eq - m), C(u) = M_g(u) M(0)^T, solved in the
 * cascade order: the 2x2 system on the second-order diagonal moments (relation (casc1)),
 * the other components one after the other (relation (casc2)). Lambda is diagonal except
 * for the block [[s+, s-], [s-, s+]] on (X^2, Y^2), s+- = (s3 +- s4)/2, where s3 and s4 are
 * the rates of X^2+Y^2 and X^2-Y^2 (s given in the order of orc_collide_geier). */
int orc_collide_cascaded(const double* f, double l, const double* s, double* fstar) {
    static const int MI[Q][Q] = {
        { 1,  1,  1,  1,  1,  1,  1,  1,  1},
        { 0,  1,  0, -1,  0,  1, -1, -1,  1},
        { 0,  0,  1,  0, -1,  1,  1, -1, -1},
        {-4, -1, -1, -1, -1,  2,  2,  2,  2},
        { 0,  1, -1,  1, -1,  0,  0,  0,  0},
        { 0,  0,  0,  0,  0,  1, -1,  1, -1},
        { 0, -2,  0,  2,  0,  1, -1, -1,  1},
        { 0,  0, -2,  0,  2,  1,  1, -1, -1},
        { 4, -2, -2, -2, -2,  1,  1,  1,  1}};
    double rho = 0.0, qx = 0.0, qy = 0.0;
    for (int j = 0; j < Q; ++j) {
        rho += f[j];
        qx += l * CX[j] * f[j];
        qy += l * CY[j] * f[j];
    }
    const double ux = qx / rho, uy = qy / rho;
    double feq[Q];
    orc_feq_product(rho, ux, uy, l, feq);
    /* Geier's original moments shifted by u */
    double Mg[Q][Q], m[Q], meq[Q];
    for (int j = 0; j < Q; ++j) {
        const double X = l * CX[j] - ux, Y = l * CY[j] - uy;
        const double l2 = l * l, l3 = l2 * l, l4 = l2 * l2;
        const double p[Q] = {1.0, X, Y, X * X / l2, Y * Y / l2, X * Y / l2, X * Y * Y / l3,
                             X * X * Y / l3, X * X * Y * Y / l4};
        for (int k = 0; k < Q; ++k) Mg[k][j] = p[k];
    }
    for (int k = 0; k < Q; ++k) {
        double a = 0.0, b = 0.0;
        for (int j = 0; j < Q; ++j) {
            a += Mg[k][j] * f[j];
            b += Mg[k][j] * feq[j];
        }
        m[k] = a;
        meq[k] = b;
    }
    /* right-hand side Lambda (m_eq - m) */
    const double sp = 0.5 * (s[3] + s[4]), sm = 0.5 * (s[3] - s[4]);
    double rhs[Q];
    for (int k = 0; k < Q; ++k) rhs[k] = 0.0;
    rhs[3] = sp * (meq[3] - m[3]) + sm * (meq[4] - m[4]);
    rhs[4] = sm * (meq[3] - m[3]) + sp * (meq[4] - m[4]);
    for (int k = 5; k < Q; ++k) rhs[k] = s[k] * (meq[k] - m[k]);
    /* C(u) = M_g(u) M(0)^T (rows of M(0) with lambda on rows 1, 2) */
    double C[Q][Q];
    for (int k = 0; k < Q; ++k)
        for (int c = 0; c < Q; ++c) {
            double a = 0.0;
            const double scale = (c == 1 || c == 2) ? l : 1.0;
            for (int j = 0; j < Q; ++j) a += Mg[k][j] * scale * MI[c][j];
            C[k][c] = a;
        }
    /* cascade: g_0 = g_1 = g_2 = 0 (conserved moments do not change); then the 2x2 block of
     * rows 3, 4 in the unknowns g_3, g_4; then rows 5..8, each solved for g_k using the
     * components already known. The system is lower triangular apart from that block. */
    double g[Q] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    {
        const double a = C[3][3], b = C[3][4], c = C[4][3], d = C[4][4];
        const double det = a * d - b * c;
        if (det == 0.0) return -1;
        g[3] = (d * rhs[3] - b * rhs[4]) / det;
        g[4] = (a * rhs[4] - c * rhs[3]) / det;
    }
    for (int k = 5; k < Q; ++k) {
        double acc = rhs[k];
        for (int c = 3; c < k; ++c) acc -= C[k][c] * g[c];
        if (C[k][k] == 0.0) return -1;
        g[k] = acc / C[k][k];
    }
    for (int j = 0; j < Q; ++j) {
        double a = 0.0;
        for (int c = 0; c < Q; ++c) {
            const double scale = (c == 1 || c == 2) ? l : 1.0;
            a += scale * MI[c][j] * g[c];
        }
        fstar[j] = f[j] + a;
    }
    return 0;
}

void orc_init_equilibrium_product(int64_t nx, int64_t ny, double l, const double* rho,
                                  const double* ux, const double* uy, double* f) {
    int64_t n = nx * ny;
    for (int64_t i = 0; i < n; ++i) {
        double feq[Q];
        orc_feq_product(rho[i], ux[i], uy[i], l, feq);
        for (int j = 0; j < Q; ++j) f[j * n + i] = feq[j];
    }
}
