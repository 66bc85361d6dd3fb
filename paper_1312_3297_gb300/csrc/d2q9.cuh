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
    const float* ut0;    // prescribed base field [2][n] or nullptr
    const float* sin_x;  // sin(2 pi x / nx), x < nx: y-component of the analytic field
};

// Modes of u~ (kernel template parameter).
enum { UM_ZERO = 0, UM_FLUID = 1, UM_ANALYTIC = 2, UM_FIELD = 3 };

// Correctly rounded reciprocal (the same value as 1.0f / x, without the division sequence).
LBMRV_HD float recip(float x) {
#ifdef __CUDA_ARCH__
    return __frcp_rn(x);
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
    return __bfloat162float(v);
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

// The relaxation of Section 1.2 in the shifted form of Section 1.3, in place on the
// deviations g of one node, for a relative velocity (ux, uy) = u~ / lambda.
//
// Since the conserved moments of d = m(0) - m_eq(0) vanish and T(u~) is lower
// block-triangular with unit diagonal blocks, only the 6x6 non-conserved block of
// T(u~) acts: identity on (e, p_xx, p_xy) plus C3 (rows q_x, q_y), D3 and D4 (row eps)
// of Appendix A. Then f* = f - M(0)^{-1} T(-u~) S T(u~) d, where M(0)^{-1} =
// M(0)^T diag(1/|row|^2) with |row|^2 = 36, 4, 4, 12, 12, 36 on the six moments.
LBMRV_HD void relax_node(float g[9], float ux, float uy, const Rates& s,
                         const StoreRef& ref) {
    const NodeMoments mo = node_moments(g);
    const float rho = ref.rho + mo.drho;
    const float ir = recip(rho);
    const float jx = ref.jx + mo.jx, jy = ref.jy + mo.jy;
    const float jxx = jx * jx * ir, jyy = jy * jy * ir;
    const float jj3 = 3.0f * (jxx + jyy);

    const float s1 = (g[1] + g[2]) + (g[3] + g[4]);
    const float s2 = (g[5] + g[6]) + (g[7] + g[8]);
    const float a = g[5] - g[7], b = g[6] - g[8];

    // d = m(0) - m_eq(0) on the non-conserved moments (Lallemand-Luo equilibrium
    // moments of the second-order polynomial equilibrium, written for deviations from
    // the reference state; see StoreRef).
    const float d_e = (-4.0f * g[0] - s1 + 2.0f * s2) + ref.c[0] + 2.0f * mo.drho - jj3;
    const float d_pxx = ((g[1] + g[3]) - (g[2] + g[4])) + ref.c[1] - (jxx - jyy);
    const float d_pxy = ((g[5] + g[7]) - (g[6] + g[8])) + ref.c[2] - jx * jy * ir;
    const float d_qx = (-2.0f * (g[1] - g[3]) + (a - b)) + ref.c[3] + jx;
    const float d_qy = (-2.0f * (g[2] - g[4]) + (a + b)) + ref.c[4] + jy;
    const float d_eps = (4.0f * g[0] - 2.0f * s1 + s2) + ref.c[5] - mo.drho + jj3;

    // Shift-block coefficients (Appendix A, blocks C3, D3, D4) at u~/lambda.
    const float ux2 = ux * ux, uy2 = uy * uy, uxy = ux * uy;
    const float d3e = 6.0f * (ux2 + uy2), d3xx = 9.0f * (ux2 - uy2), d3xy = 36.0f * uxy;

    // Forward shift T(u~) d, then the diagonal relaxation S.
    const float t_qx = d_qx - 2.0f * ux * d_e - 3.0f * ux * d_pxx - 6.0f * uy * d_pxy;
    const float t_qy = d_qy - 2.0f * uy * d_e + 3.0f * uy * d_pxx - 6.0f * ux * d_pxy;
    const float t_eps = d_eps + d3e * d_e + d3xx * d_pxx + d3xy * d_pxy - 6.0f * ux * d_qx -
                        6.0f * uy * d_qy;
    const float r_e = s.e * d_e, r_pxx = s.pxx * d_pxx, r_pxy = s.pxy * d_pxy;
    const float r_qx = s.qx * t_qx, r_qy = s.qy * t_qy, r_eps = s.eps * t_eps;

    // Back shift T(-u~) (morphism: T(u~)^{-1} = T(-u~)).
    const float h_qx = r_qx + 2.0f * ux * r_e + 3.0f * ux * r_pxx + 6.0f * uy * r_pxy;
    const float h_qy = r_qy + 2.0f * uy * r_e - 3.0f * uy * r_pxx + 6.0f * ux * r_pxy;
    const float h_eps = r_eps + d3e * r_e + d3xx * r_pxx + d3xy * r_pxy + 6.0f * ux * r_qx +
                        6.0f * uy * r_qy;

    // f* = f - M(0)^{-1} h.
    const float ce = r_e * (1.0f / 36.0f), cxx = r_pxx * 0.25f, cxy = r_pxy * 0.25f;
    const float cqx = h_qx * (1.0f / 12.0f), cqy = h_qy * (1.0f / 12.0f);
    const float cep = h_eps * (1.0f / 36.0f);
    const float axis_c = -ce - 2.0f * cep;       // common to j = 1..4
    const float diag_c = 2.0f * ce + cep;        // common to j = 5..8
    g[0] -= -4.0f * ce + 4.0f * cep;
    g[1] -= axis_c + cxx - 2.0f * cqx;
    g[2] -= axis_c - cxx - 2.0f * cqy;
    g[3] -= axis_c + cxx + 2.0f * cqx;
    g[4] -= axis_c - cxx + 2.0f * cqy;
    g[5] -= diag_c + cxy + cqx + cqy;
    g[6] -= diag_c - cxy - cqx + cqy;
    g[7] -= diag_c + cxy - cqx - cqy;
    g[8] -= diag_c - cxy + cqx - cqy;
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
        ux = a.amp_t * cospif(a.two_over_ny * (float)y);
        uy = a.amp_t * __ldg(a.sin_x + x);
    } else {
        const int64_t n = (int64_t)a.nx * a.ny;
        ux = a.amp_t * __ldg(a.ut0 + i);
        uy = a.amp_t * __ldg(a.ut0 + n + i);
    }
}

}  // namespace lbmrv
