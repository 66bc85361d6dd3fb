/*
 * FP64 CPU oracle for the relative-velocity scheme on a periodic D3Q19 lattice.
 *
 * TEST INFRASTRUCTURE, like lbmrv_oracle.c: loaded only by the tests, the smoke check and
 * the benchmark's CPU leg; shares nothing with the CUDA library.
 *
 * The paper (arXiv:1312.3297) defines the scheme for any DdQq (Sections 1.1 and 1.2) but
 * gives a moment basis only for D2Q9. This oracle takes Section 1.2 literally with the
 * following 3D basis (reading; see the design notes): 19 polynomials spanning the
 * translation-invariant space
 *   1, X, Y, Z, (X^2+Y^2+Z^2), (X^2-Y^2), (Y^2-Z^2), XY, XZ, YZ,
 *   XY^2, XZ^2, YX^2, YZ^2, ZX^2, ZY^2, X^2Y^2, X^2Z^2, Y^2Z^2
 * (divided by lambda^degree from degree 2 on, as the D2Q9 set of relation (mom) is). Its
 * span is closed under differentiation, so M(u~) = T(u~) M(0) with T lower triangular and
 * T(u~+v~) = T(u~) T(v~) (the condition stated after the morphism proposition of Section
 * 1.3); the usual d'Humieres D3Q19 basis does not have this property.
 *
 * Steps per node (definition): M(u~)_kj = P_k(v_j - u~) (relation (MatMu)), m = M(u~) f,
 * m_eq = M(u~) f_eq, m*_k = m_k + s_k (m_eq,k - m_k) (relation (relaxationu)),
 * f* = M(u~)^{-1} m* by LU with partial pivoting; then f_j(x, t+dt) = f*_j(x - v_j dt)
 * (relation (transport)), periodic.
 * Equilibrium (reading): second-order polynomial D3Q19 equilibrium, w = 1/3 (rest),
 * 1/18 (faces), 1/36 (edges), c_s^2 = lambda^2 / 3. Lattice units dx = 1.
 * Layout: f[((j*nz + z)*ny + y)*nx + x].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define Q3 19

static const int CX3[Q3] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int CY3[Q3] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int CZ3[Q3] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};

void orc3_velocities(int* cx, int* cy, int* cz) {
    for (int j = 0; j < Q3; ++j) {
        cx[j] = CX3[j];
        cy[j] = CY3[j];
        cz[j] = CZ3[j];
    }
}

/* The 19 basis polynomials at (X, Y, Z). */
double orc3_poly(int k, double X, double Y, double Z, double l) {
    double l2 = l * l, l3 = l2 * l, l4 = l2 * l2;
    switch (k) {
        case 0: return 1.0;
        case 1: return X;
        case 2: return Y;
        case 3: return Z;
        case 4: return (X * X + Y * Y + Z * Z) / l2;
        case 5: return (X * X - Y * Y) / l2;
        case 6: return (Y * Y - Z * Z) / l2;
        case 7: return X * Y / l2;
        case 8: return X * Z / l2;
        case 9: return Y * Z / l2;
        case 10: return X * Y * Y / l3;
        case 11: return X * Z * Z / l3;
        case 12: return Y * X * X / l3;
        case 13: return Y * Z * Z / l3;
        case 14: return Z * X * X / l3;
        case 15: return Z * Y * Y / l3;
        case 16: return X * X * Y * Y / l4;
        case 17: return X * X * Z * Z / l4;
        case 18: return Y * Y * Z * Z / l4;
        default: return NAN;
    }
}

void orc3_moment_matrix(double ux, double uy, double uz, double l, double* M) {
    for (int k = 0; k < Q3; ++k)
        for (int j = 0; j < Q3; ++j)
            M[k * Q3 + j] = orc3_poly(k, l * CX3[j] - ux, l * CY3[j] - uy, l * CZ3[j] - uz, l);
}

void orc3_feq(double rho, double ux, double uy, double uz, double l, double* feq) {
    double l2 = l * l;
    double uu = ux * ux + uy * uy + uz * uz;
    for (int j = 0; j < Q3; ++j) {
        int nnz = (CX3[j] != 0) + (CY3[j] != 0) + (CZ3[j] != 0);
        double w = nnz == 0 ? 1.0 / 3.0
                            : (nnz == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
        double vu = l * (CX3[j] * ux + CY3[j] * uy + CZ3[j] * uz);
        feq[j] = w * rho * (1.0 + 3.0 * vu / l2 + 4.5 * vu * vu / (l2 * l2) - 1.5 * uu / l2);
    }
}

static int lu_solve19(double* A, double* b, double* x) {
    for (int c = 0; c < Q3; ++c) {
        int p = c;
        double best = fabs(A[c * Q3 + c]);
        for (int r = c + 1; r < Q3; ++r) {
            double v = fabs(A[r * Q3 + c]);
            if (v > best) { best = v; p = r; }
        }
        if (best == 0.0) return -1;
        if (p != c) {
            for (int k = 0; k < Q3; ++k) {
                double t = A[c * Q3 + k]; A[c * Q3 + k] = A[p * Q3 + k]; A[p * Q3 + k] = t;
            }
            double t = b[c]; b[c] = b[p]; b[p] = t;
        }
        for (int r = c + 1; r < Q3; ++r) {
            double m = A[r * Q3 + c] / A[c * Q3 + c];
            for (int k = c; k < Q3; ++k) A[r * Q3 + k] -= m * A[c * Q3 + k];
            b[r] -= m * b[c];
        }
    }
    for (int r = Q3 - 1; r >= 0; --r) {
        double acc = b[r];
        for (int k = r + 1; k < Q3; ++k) acc -= A[r * Q3 + k] * x[k];
        x[r] = acc / A[r * Q3 + r];
    }
    return 0;
}

static void conserved3(const double* f, double l, double* rho, double* q) {
    double r = 0.0, a = 0.0, b = 0.0, c = 0.0;
    for (int j = 0; j < Q3; ++j) {
        r += f[j];
        a += l * CX3[j] * f[j];
        b += l * CY3[j] * f[j];
        c += l * CZ3[j] * f[j];
    }
    *rho = r;
    q[0] = a;
    q[1] = b;
    q[2] = c;
}

/* One relaxation at a node (Section 1.2 as defined). Returns 0 or -1 (singular). */
int orc3_collide_node(const double* f, const double* ut, double l, const double* s,
                      double* fstar) {
    double M[Q3 * Q3], feq[Q3], m[Q3], meq[Q3], ms[Q3], rho, q[3];
    conserved3(f, l, &rho, q);
    orc3_feq(rho, q[0] / rho, q[1] / rho, q[2] / rho, l, feq);
    orc3_moment_matrix(ut[0], ut[1], ut[2], l, M);
    for (int k = 0; k < Q3; ++k) {
        double a = 0.0, b = 0.0;
        for (int j = 0; j < Q3; ++j) {
            a += M[k * Q3 + j] * f[j];
            b += M[k * Q3 + j] * feq[j];
        }
        m[k] = a;
        meq[k] = b;
    }
    for (int k = 0; k < Q3; ++k) ms[k] = m[k] + s[k] * (meq[k] - m[k]);
    return lu_solve19(M, ms, fstar);
}

/* Relaxation at every node at time t; mode 0: u~ = 0, 1: u~ = q/rho, 2: prescribed
 * u~ = amp * ut0(x) * cos(2 pi t / period) with ut0[3][n] (required). */
int orc3_collide_lattice(int64_t nx, int64_t ny, int64_t nz, double l, const double* s,
                         int mode, const double* ut0, double amp, double period, int64_t t,
                         const double* fin, double* fout, int nthreads) {
    int64_t n = nx * ny * nz;
    int status = 0;
    double tf = 1.0;
    if (mode == 2 && period > 0.0) tf = cos(6.283185307179586476925286766559 * (double)t / period);
    if (mode == 2 && !ut0) return -2;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(static) num_threads(nthreads) reduction(min : status)
    for (int64_t i = 0; i < n; ++i) {
        double f[Q3], fs[Q3], ut[3] = {0.0, 0.0, 0.0};
        for (int j = 0; j < Q3; ++j) f[j] = fin[j * n + i];
        if (mode == 1) {
            double rho, q[3];
            conserved3(f, l, &rho, q);
            for (int a = 0; a < 3; ++a) ut[a] = q[a] / rho;
        } else if (mode == 2) {
            for (int a = 0; a < 3; ++a) ut[a] = amp * ut0[a * n + i] * tf;
        }
        if (orc3_collide_node(f, ut, l, s, fs) != 0) status = -1;
        for (int j = 0; j < Q3; ++j) fout[j * n + i] = fs[j];
    }
    return status;
}

void orc3_stream(int64_t nx, int64_t ny, int64_t nz, const double* fin, double* fout,
                 int nthreads) {
    int64_t n = nx * ny * nz;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x)
                for (int j = 0; j < Q3; ++j) {
                    int64_t xs = ((x - CX3[j]) % nx + nx) % nx;
                    int64_t ys = ((y - CY3[j]) % ny + ny) % ny;
                    int64_t zs = ((z - CZ3[j]) % nz + nz) % nz;
                    fout[j * n + (z * ny + y) * nx + x] = fin[j * n + (zs * ny + ys) * nx + xs];
                }
}

int orc3_run(int64_t nx, int64_t ny, int64_t nz, double l, const double* s, int mode,
             const double* ut0, double amp, double period, int64_t t0, int64_t nsteps,
             double* f, double* work, int nthreads) {
    for (int64_t k = 0; k < nsteps; ++k) {
        int rc = orc3_collide_lattice(nx, ny, nz, l, s, mode, ut0, amp, period, t0 + k, f, work,
                                      nthreads);
        if (rc != 0) return rc;
        orc3_stream(nx, ny, nz, work, f, nthreads);
    }
    return 0;
}

void orc3_init_equilibrium(int64_t n, double l, const double* rho, const double* u, double* f) {
    for (int64_t i = 0; i < n; ++i) {
        double feq[Q3];
        orc3_feq(rho[i], u[i], u[n + i], u[2 * n + i], l, feq);
        for (int j = 0; j < Q3; ++j) f[j * n + i] = feq[j];
    }
}

void orc3_moments(int64_t n, double l, const double* f, double* rho, double* u) {
    for (int64_t i = 0; i < n; ++i) {
        double g[Q3], r, q[3];
        for (int j = 0; j < Q3; ++j) g[j] = f[j * n + i];
        conserved3(g, l, &r, q);
        rho[i] = r;
        for (int a = 0; a < 3; ++a) u[a * n + i] = q[a] / r;
    }
}
