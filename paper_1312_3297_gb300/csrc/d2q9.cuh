// D2Q9 relative-velocity lattice Boltzmann: device-side pieces shared by the kernels.
//
// Notation (Section 1.3 of arXiv:1312.3297): velocities c_j = v_j / lambda in the order
// (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),(-1,-1),(1,-1); moments in the order
// rho, q_x, q_y, e, p_xx, p_xy, q_x(3rd), q_y(3rd), eps of relation (mom). With
// lattice-normalised velocities everything below is lambda-free except u~ / lambda.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <cmath>

#ifdef __CUDACC__
#include "f32x2.cuh"
#endif

#define LBMRV_HD __host__ __device__ __forceinline__

namespace lbmrv {

// Rates on the six non-conserved moments (e, p_xx, p_xy, q_x, q_y, eps).
struct Rates {
    float e, pxx, pxy, qx, qy, eps;
};

// Reference state of the stored deviations g = f - f_eq(rho_ref, U_ref), in lattice
// units (velocities divided by lambda): rho, the reference momentum j = rho_ref U, the
// reference velocity U, and c = M(0) f_eq(rho_ref, U) - m_eq(0)(rho_ref, j) + (2 rho_ref,
// 0, 0, 0, 0, -rho_ref) on the six non-conserved moments, i.e. the constant part of
// d = m(0) - m_eq(0) once the deviation sums are split off. U = 0 gives j = c = 0.
struct StoreRef {
    float rho;
    float jx, jy;
    float ux, uy;
    float c[6];
};

// Per-launch arguments of the fused step.
struct StepArgs {
    int nx, ny;
    Rates s;
    StoreRef ref;        // stored value g = f - f_eq(ref)
    float amp_t;         // prescribed mode: A cos(2 pi t / P) / lambda at this step
    float two_over_nx;   // 2 / nx, 2 / ny for cospi/sinpi of the analytic field
    float two_over_ny;
    int y_off;           // global row of local row y is y + y_off (a slab; else 0)
    const float* ut0;    // prescribed base field [2][n] or nullptr
    const float* sin_x;  // sin(2 pi x / nx), x < nx: y-component of the analytic field
};

// Modes of u~ (kernel template parameter).
enum { UM_ZERO = 0, UM_FLUID = 1, UM_ANALYTIC = 2, UM_FIELD = 3 };

// Reciprocal of a density (close to 1) on the device, in one of three forms of the same
// accuracy class: the hardware approximation (rcp.approx.ftz.f32, at most 1 ulp from 1/x
// per the PTX ISA), the fast division intrinsic (at most 2 ulp) and the correctly rounded
// reciprocal. For densities near 1 (no subnormals, no overflow) all three serve; they
// differ in the instructions around the special-function unit and therefore in how the
// compiler schedules a whole step, so each step kernel names the form measured fastest
// for it. Plain division on the host.
enum { RCP_APPROX = 0, RCP_DIV = 1, RCP_RN = 2 };

template <int RCP = RCP_RN>
LBMRV_HD float recip(float x) {
#ifdef __CUDA_ARCH__
    if constexpr (RCP == RCP_APPROX) {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    } else if constexpr (RCP == RCP_DIV) {
        return __fdividef(1.0f, x);
    } else {
        return __frcp_rn(x);
    }
#else
    return 1.0f / x;
#endif
}

LBMRV_HD float wgt(int j) {
    return j == 0 ? (4.0f / 9.0f) : (j < 5 ? (1.0f / 9.0f) : (1.0f / 36.0f));
}

template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) {
    return __uint_as_float((uint32_t)__bfloat16_as_ushort(v) << 16);  // the upper half
}

template <typename T> __device__ __forceinline__ T from_f(float v);
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <> __device__ __forceinline__ __half from_f<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}

// Sums of the stored deviations g of one node: rho = rho_ref + drho, q / lambda =
// j_ref + (jx, jy).
struct NodeMoments {
    float drho;  // sum g
    float jx, jy;  // sum c g
};

LBMRV_HD NodeMoments node_moments(const float g[9]) {
    NodeMoments m;
    const float a = g[5] - g[7], b = g[6] - g[8];
    m.drho = ((g[0] + (g[1] + g[2]) + (g[3] + g[4])) + ((g[5] + g[6]) + (g[7] + g[8])));
    m.jx = (g[1] - g[3]) + (a - b);
    m.jy = (g[2] - g[4]) + (a + b);
    return m;
}

LBMRV_HD float fma_(float a, float b, float c) { return fmaf(a, b, c); }

// x is neither infinite nor NaN. On the device an integer test of the exponent bits, so
// that no FP64 instruction is involved (FP64 issues at 2 operations per clock per SM on
// this GPU).
LBMRV_HD bool finite_f(float x) {
#ifdef __CUDA_ARCH__
    return (__float_as_uint(x) & 0x7f800000u) != 0x7f800000u;
#else
    return std::isfinite(x);
#endif
}

#ifdef __CUDACC__
// Lane-wise reciprocal of a pair of densities.
template <int RCP = RCP_RN>
__device__ __forceinline__ F2 recip(F2 x) {
    float a, b;
    unpack2(x, a, b);
    return pack2(recip<RCP>(a), recip<RCP>(b));
}

template <int RCP = RCP_RN>
__device__ __forceinline__ F1 recip(F1 x) {
    return F1(recip<RCP>(x.v));
}
#endif

// The relaxation of Section 1.2 in the shifted form of Section 1.3, in place on the
// deviations g of one node (R = float) or of two nodes at once (R = F2, one node per
// lane), for a relative velocity (ux, uy) = u~ / lambda. UM = UM_FLUID takes u~ = q / rho
// of the state being relaxed (ux, uy are outputs then); UM = UM_ZERO is the fixed-frame
// MRT scheme (ux, uy ignored). RCP: the form of 1/rho (see recip).
//
// Since the conserved moments of d = m(0) - m_eq(0) vanish and T(u~) is lower
// block-triangular with unit diagonal blocks, only the 6x6 non-conserved block of
// T(u~) acts: identity on (e, p_xx, p_xy) plus C3 (rows q_x, q_y), D3 and D4 (row eps)
// of Appendix A. Then f* = f - M(0)^{-1} T(-u~) S T(u~) d, where M(0)^{-1} =
// M(0)^T diag(1/|row|^2) with |row|^2 = 36, 4, 4, 12, 12, 36 on the six moments.
template <int UM, int RCP = RCP_RN, typename R>
LBMRV_HD void relax_node(R g[9], R& ux, R& uy, const Rates& s, const StoreRef& ref) {
    // Sums and differences of opposite populations.
    const R a1 = g[1] + g[3], b1 = g[1] - g[3], a2 = g[2] + g[4], b2 = g[2] - g[4];
    const R a5 = g[5] + g[7], b5 = g[5] - g[7], a6 = g[6] + g[8], b6 = g[6] - g[8];
    const R s1 = a1 + a2, s2 = a5 + a6;
    const R bm = b5 - b6, bp = b5 + b6;
    // Conserved moments: rho = rho_ref + drho, q / lambda = j (relation (rhoq)).
    const R drho = g[0] + (s1 + s2);
    const R ir = recip<RCP>(R(ref.rho) + drho);
    const R jx = R(ref.jx) + (b1 + bm), jy = R(ref.jy) + (b2 + bp);
    const R vx = jx * ir, vy = jy * ir;  // q / (rho lambda)
    if constexpr (UM == UM_FLUID) {
        ux = vx;
        uy = vy;
    }

    // d = m(0) - m_eq(0) on (e, p_xx, p_xy, q_x, q_y, eps) for the Lallemand-Luo
    // equilibrium moments (-2 rho + 3 |j|^2 / rho, (jx^2 - jy^2) / rho, jx jy / rho, -jx,
    // -jy, rho - 3 |j|^2 / rho) of the second-order polynomial equilibrium. The rows of
    // M(0) are written through the pair sums and drho; the reference state enters through
    // ref.c (see StoreRef). In the q rows the reference terms cancel exactly.
    const R kx = jx * vx, ky = jy * vy;
    const R kin = kx + ky, kxy = kx - ky;  // |j|^2 / rho, (jx^2 - jy^2) / rho
    const R d_e = fma_(R(4.0f), s2, fma_(R(-2.0f), g[0], s1)) - fma_(R(3.0f), kin, R(-ref.c[0]));
    const R d_pxx = (a1 - a2) - (kxy - R(ref.c[1]));
    const R d_pxy = (a5 - a6) - fma_(jx, vy, R(-ref.c[2]));
    const R d_qx = (bm + bm) - b1;
    const R d_qy = (bp + bp) - b2;
    const R d_eps = fma_(R(3.0f), g[0] - s1, fma_(R(3.0f), kin, R(ref.c[5])));

    R h_qx, h_qy, h_eps;
    const R r_e = R(s.e) * d_e, r_pxx = R(s.pxx) * d_pxx, r_pxy = R(s.pxy) * d_pxy;
    if constexpr (UM == UM_ZERO) {
        h_qx = R(s.qx) * d_qx;
        h_qy = R(s.qy) * d_qy;
        h_eps = R(s.eps) * d_eps;
    } else {
        // Shift-block coefficients (Appendix A, blocks C3, D3, D4) at u~ / lambda.
        const R ux2 = ux + ux, uy2 = uy + uy, ux3 = ux2 + ux, uy3 = uy2 + uy;
        const R ux6 = ux3 + ux3, uy6 = uy3 + uy3;
        const R d3e = fma_(ux6, ux, uy6 * uy);       // 6 |u|^2
        const R d3xx = ux3 * ux3 - uy3 * uy3;        // 9 (ux^2 - uy^2)
        const R d3xy = ux6 * uy6;                    // 36 ux uy
        // Forward shift T(u~) d, then the diagonal relaxation S.
        const R t_qx = d_qx - fma_(ux2, d_e, fma_(ux3, d_pxx, uy6 * d_pxy));
        const R t_qy = fma_(uy3, d_pxx, d_qy) - fma_(uy2, d_e, ux6 * d_pxy);
        const R t_eps = fma_(d3e, d_e, fma_(d3xx, d_pxx, fma_(d3xy, d_pxy, d_eps))) -
                        fma_(ux6, d_qx, uy6 * d_qy);
        const R r_qx = R(s.qx) * t_qx, r_qy = R(s.qy) * t_qy, r_eps = R(s.eps) * t_eps;
        // Back shift T(-u~) (morphism: T(u~)^{-1} = T(-u~)).
        h_qx = fma_(ux2, r_e, fma_(ux3, r_pxx, fma_(uy6, r_pxy, r_qx)));
        h_qy = fma_(uy2, r_e, fma_(ux6, r_pxy, r_qy)) - uy3 * r_pxx;
        h_eps = fma_(d3e, r_e, fma_(d3xx, r_pxx, fma_(d3xy, r_pxy,
                    fma_(ux6, r_qx, fma_(uy6, r_qy, r_eps)))));
    }

    // f* = f - M(0)^{-1} h, M(0)^{-1} = M(0)^T diag(1/36, 1/4, 1/4, 1/12, 1/12, 1/36) on
    // (e, p_xx, p_xy, q_x, q_y, eps), with the shared sums of the nine columns factored.
    const R rest = (h_eps - r_e) * R(1.0f / 9.0f);                           // j = 0
    const R axis = fma_(h_eps, R(-2.0f / 36.0f), r_e * R(-1.0f / 36.0f));    // j = 1..4
    const R diag = fma_(r_e, R(2.0f / 36.0f), h_eps * R(1.0f / 36.0f));      // j = 5..8
    const R ax_p = fma_(R(0.25f), r_pxx, axis), ax_m = fma_(R(-0.25f), r_pxx, axis);
    const R dg_p = fma_(R(0.25f), r_pxy, diag), dg_m = fma_(R(-0.25f), r_pxy, diag);
    const R hs = h_qx + h_qy, hd = h_qx - h_qy;
    g[0] = g[0] - rest;
    g[1] = fma_(h_qx, R(1.0f / 6.0f), g[1] - ax_p);
    g[3] = fma_(h_qx, R(-1.0f / 6.0f), g[3] - ax_p);
    g[2] = fma_(h_qy, R(1.0f / 6.0f), g[2] - ax_m);
    g[4] = fma_(h_qy, R(-1.0f / 6.0f), g[4] - ax_m);
    g[5] = fma_(hs, R(-1.0f / 12.0f), g[5] - dg_p);
    g[7] = fma_(hs, R(1.0f / 12.0f), g[7] - dg_p);
    g[6] = fma_(hd, R(1.0f / 12.0f), g[6] - dg_m);
    g[8] = fma_(hd, R(-1.0f / 12.0f), g[8] - dg_m);
}

// u~ / lambda at node (x, y) for the compile-time mode.
template <int UM>
__device__ __forceinline__ void relative_velocity(const float g[9], const StoreRef& ref, int x,
                                                  int y, int64_t i, const StepArgs& a,
                                                  float& ux, float& uy) {
    if (UM == UM_ZERO) {
        ux = 0.0f;
        uy = 0.0f;
    } else if (UM == UM_FLUID) {
        const NodeMoments m = node_moments(g);
        const float ir = recip(ref.rho + m.drho);
        ux = (ref.jx + m.jx) * ir;
        uy = (ref.jy + m.jy) * ir;
    } else if (UM == UM_ANALYTIC) {
        ux = a.amp_t * cospif(a.two_over_ny * (float)(y + a.y_off));
        uy = a.amp_t * __ldg(a.sin_x + x);
    } else {
        const int64_t n = (int64_t)a.nx * a.ny;
        ux = a.amp_t * __ldg(a.ut0 + i);
        uy = a.amp_t * __ldg(a.ut0 + n + i);
    }
}

}  // namespace lbmrv

namespace lbmrv {

// Geier's cascaded scheme as a scheme with relative velocities (the proposition of Section
// 1.3 on the cascaded scheme, Appendix B): D2Q9 with the basis 1, X, Y, X^2+Y^2, X^2-Y^2,
// XY, XY^2, X^2Y, X^2Y^2 (relation (polgeier)) and the product-form equilibrium, whose
// moments in the frame of the fluid velocity are those of the Maxwellian. Rates (Rates
// fields reused): e = X^2+Y^2, pxx = X^2-Y^2, pxy = XY, qx = XY^2, qy = X^2Y, eps = X^2Y^2.
// The non-conserved moments are handled as monomials XX, YY, XY, XYY, YXX, XXYY; ref.c
// holds the constant parts (XX, YY, XY, XYY, YXX, XXYY) of the reference equilibrium.
LBMRV_HD void relax_node_geier(float g[9], float ux, float uy, const Rates& s,
                               const StoreRef& ref) {
    const NodeMoments mo = node_moments(g);
    const float ir = recip(ref.rho + mo.drho);
    const float jx = ref.jx + mo.jx, jy = ref.jy + mo.jy;
    const float vx = jx * ir, vy = jy * ir;  // fluid velocity (equilibrium)
    const float third = 1.0f / 3.0f;
    const float dsum = (g[5] + g[6]) + (g[7] + g[8]);
    // d = m(0) - m_eq(0) on the raw monomials; product equilibrium:
    // XX: rho/3 + rho vx^2, XY: rho vx vy, XYY: rho vx (1/3 + vy^2),
    // XXYY: rho (1/3 + vx^2)(1/3 + vy^2).
    const float d_xx = ((g[1] + g[3]) + dsum) - third * mo.drho + ref.c[0] - jx * vx;
    const float d_yy = ((g[2] + g[4]) + dsum) - third * mo.drho + ref.c[1] - jy * vy;
    const float d_xy = ((g[5] + g[7]) - (g[6] + g[8])) + ref.c[2] - jx * vy;
    const float d_xyy = ((g[5] - g[7]) + (g[8] - g[6])) - third * mo.jx + ref.c[3] - jx * vy * vy;
    const float d_yxx = ((g[5] - g[7]) + (g[6] - g[8])) - third * mo.jy + ref.c[4] - jy * vx * vx;
    const float d_xxyy = dsum - (1.0f / 9.0f) * mo.drho + ref.c[5] -
                         (third * (jx * vx + jy * vy) + jx * vx * vy * vy);
    // shift to the frame moving at u~ (binomial expansion; lower non-conserved orders only)
    const float k_xyy = d_xyy - 2.0f * uy * d_xy - ux * d_yy;
    const float k_yxx = d_yxx - 2.0f * ux * d_xy - uy * d_xx;
    const float k_xxyy = d_xxyy - 2.0f * uy * d_yxx - 2.0f * ux * d_xyy + uy * uy * d_xx +
                         ux * ux * d_yy + 4.0f * ux * uy * d_xy;
    // relaxation, diagonal in X^2+Y^2, X^2-Y^2, XY, XY^2, X^2Y, X^2Y^2
    const float rt = s.e * (d_xx + d_yy), rd = s.pxx * (d_xx - d_yy);
    const float r_xx = 0.5f * (rt + rd), r_yy = 0.5f * (rt - rd);
    const float r_xy = s.pxy * d_xy;
    const float r_xyy = s.qx * k_xyy, r_yxx = s.qy * k_yxx, r_xxyy = s.eps * k_xxyy;
    // back to the fixed frame
    const float h_xyy = r_xyy + 2.0f * uy * r_xy + ux * r_yy;
    const float h_yxx = r_yxx + 2.0f * ux * r_xy + uy * r_xx;
    const float h_xxyy = r_xxyy + 2.0f * uy * r_yxx + 2.0f * ux * r_xyy + uy * uy * r_xx +
                         ux * ux * r_yy + 4.0f * ux * uy * r_xy;
    // populations of the increment (monomial moments with zero conserved part)
    const float pd = 0.5f * (h_xxyy + r_xy), qd = 0.5f * (h_xxyy - r_xy);
    const float r1 = 0.5f * (h_xyy + h_yxx), r2 = 0.5f * (h_xyy - h_yxx);
    g[5] -= 0.5f * (pd + r1);
    g[7] -= 0.5f * (pd - r1);
    g[8] -= 0.5f * (qd + r2);
    g[6] -= 0.5f * (qd - r2);
    const float ax = r_xx - h_xxyy, ay = r_yy - h_xxyy;
    g[1] -= 0.5f * (ax - h_xyy);
    g[3] -= 0.5f * (ax + h_xyy);
    g[2] -= 0.5f * (ay - h_yxx);
    g[4] -= 0.5f * (ay + h_yxx);
    g[0] -= h_xxyy - (r_xx + r_yy);
}

// The same relaxation on one node (R = F1) or two nodes at once (R = F2, one per lane,
// packed FP32 instructions), with every fused multiply-add written out; UM = UM_FLUID takes
// u~ = q / rho of the node being relaxed (ux, uy ignored), UM = UM_ZERO skips the shift.
template <int UM, int RCP, typename R>
LBMRV_HD void relax_node_geier_r(R g[9], R ux, R uy, const Rates& s, const StoreRef& ref) {
    const R a = g[5] - g[7], b = g[6] - g[8];
    const R dsum = (g[5] + g[6]) + (g[7] + g[8]);
    const R drho = ((g[0] + (g[1] + g[2])) + (g[3] + g[4])) + dsum;
    const R mjx = (g[1] - g[3]) + (a - b), mjy = (g[2] - g[4]) + (a + b);
    const R ir = recip<RCP>(R(ref.rho) + drho);
    const R jx = R(ref.jx) + mjx, jy = R(ref.jy) + mjy;
    const R vx = jx * ir, vy = jy * ir;  // fluid velocity (equilibrium)
    if constexpr (UM == UM_FLUID) {
        ux = vx;
        uy = vy;
    }
    const R third = R(1.0f / 3.0f);
    const R kx = jx * vx, ky = jy * vy;  // jx^2 / rho, jy^2 / rho
    // d = m(0) - m_eq(0) on the monomials, product equilibrium (see relax_node_geier)
    const R d_xx = (((g[1] + g[3]) + dsum) + R(ref.c[0])) - fma_(third, drho, kx);
    const R d_yy = (((g[2] + g[4]) + dsum) + R(ref.c[1])) - fma_(third, drho, ky);
    const R pxy = jx * vy;               // jx jy / rho
    const R d_xy = (((g[5] + g[7]) - (g[6] + g[8])) + R(ref.c[2])) - pxy;
    const R d_xyy = ((a - b) + R(ref.c[3])) - fma_(third, mjx, pxy * vy);
    const R d_yxx = ((a + b) + R(ref.c[4])) - fma_(third, mjy, pxy * vx);
    const R d_xxyy = (dsum + R(ref.c[5])) -
                     fma_(R(1.0f / 9.0f), drho, fma_(third, kx + ky, kx * (vy * vy)));
    R k_xyy = d_xyy, k_yxx = d_yxx, k_xxyy = d_xxyy;
    R ux2 = R(0.0f), uy2 = R(0.0f), uxx = R(0.0f), uyy = R(0.0f), uxy4 = R(0.0f);
    if constexpr (UM != UM_ZERO) {  // shift to the frame moving at u~
        ux2 = ux + ux;
        uy2 = uy + uy;
        uxx = ux * ux;
        uyy = uy * uy;
        uxy4 = ux2 * uy2;
        k_xyy = d_xyy - fma_(uy2, d_xy, ux * d_yy);
        k_yxx = d_yxx - fma_(ux2, d_xy, uy * d_xx);
        k_xxyy = fma_(uyy, d_xx, fma_(uxx, d_yy, fma_(uxy4, d_xy, d_xxyy))) -
                 fma_(uy2, d_yxx, ux2 * d_xyy);
    }
    // relaxation, diagonal in X^2+Y^2, X^2-Y^2, XY, XY^2, X^2Y, X^2Y^2
    const R half = R(0.5f);
    const R rt = R(s.e) * (d_xx + d_yy), rd = R(s.pxx) * (d_xx - d_yy);
    const R r_xx = half * (rt + rd), r_yy = half * (rt - rd);
    const R r_xy = R(s.pxy) * d_xy;
    const R r_xyy = R(s.qx) * k_xyy, r_yxx = R(s.qy) * k_yxx, r_xxyy = R(s.eps) * k_xxyy;
    R h_xyy = r_xyy, h_yxx = r_yxx, h_xxyy = r_xxyy;
    if constexpr (UM != UM_ZERO) {  // back to the fixed frame
        h_xyy = fma_(uy2, r_xy, fma_(ux, r_yy, r_xyy));
        h_yxx = fma_(ux2, r_xy, fma_(uy, r_xx, r_yxx));
        h_xxyy = fma_(uy2, r_yxx, fma_(ux2, r_xyy,
                 fma_(uyy, r_xx, fma_(uxx, r_yy, fma_(uxy4, r_xy, r_xxyy)))));
    }
    // populations of the increment (monomial moments with zero conserved part)
    const R mq = R(-0.25f);
    const R pd = h_xxyy + r_xy, qd = h_xxyy - r_xy;
    const R r1 = h_xyy + h_yxx, r2 = h_xyy - h_yxx;
    g[5] = fma_(mq, pd + r1, g[5]);
    g[7] = fma_(mq, pd - r1, g[7]);
    g[8] = fma_(mq, qd + r2, g[8]);
    g[6] = fma_(mq, qd - r2, g[6]);
    const R ax = r_xx - h_xxyy, ay = r_yy - h_xxyy;
    g[1] = fma_(R(-0.5f), ax - h_xyy, g[1]);
    g[3] = fma_(R(-0.5f), ax + h_xyy, g[3]);
    g[2] = fma_(R(-0.5f), ay - h_yxx, g[2]);
    g[4] = fma_(R(-0.5f), ay + h_yxx, g[4]);
    g[0] = g[0] - (h_xxyy - (r_xx + r_yy));
}

}  // namespace lbmrv
