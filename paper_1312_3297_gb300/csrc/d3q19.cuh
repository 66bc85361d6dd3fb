// D3Q19 relative-velocity relaxation (device side).
//
// The paper (arXiv:1312.3297) defines the scheme for any DdQq (Sections 1.1-1.2) but prints
// a basis only for D2Q9. This lattice uses 19 polynomials whose span is closed under
// differentiation, so that M(u~) = T(u~) M(0) with T lower triangular and
// T(u~)^{-1} = T(-u~), the property the shifted form of Section 1.3 needs:
//   1, X, Y, Z | X^2+Y^2+Z^2, X^2-Y^2, Y^2-Z^2, XY, XZ, YZ |
//   XY^2, XZ^2, YX^2, YZ^2, ZX^2, ZY^2 | X^2Y^2, X^2Z^2, Y^2Z^2
// (rates s[0..18] in this order). Internally the non-conserved moments are kept as
// monomials; the shift T(u~) is then the binomial expansion of (X - u~x)^a (Y - u~y)^b
// (Z - u~z)^c, which only couples lower to higher degrees. The relaxation of the second-order
// diagonal block is diagonal in (trace, X^2-Y^2, Y^2-Z^2), as the basis says.
//
// Velocities, in units of lambda: 0 (0,0,0); 1-6 (+-1,0,0), (0,+-1,0), (0,0,+-1);
// 7-10 (1,1,0), (-1,-1,0), (1,-1,0), (-1,1,0); 11-14 (1,0,1), (-1,0,-1), (1,0,-1), (-1,0,1);
// 15-18 (0,1,1), (0,-1,-1), (0,1,-1), (0,-1,1).
#pragma once

#include "d2q9.cuh"

namespace lbmrv {

// Rates on the 15 non-conserved basis polynomials (s[4..18] of the API).
struct Rates3 {
    float e, a, b, xy, xz, yz;                // trace, X^2-Y^2, Y^2-Z^2, XY, XZ, YZ
    float xyy, xzz, yxx, yzz, zxx, zyy;       // third order
    float xxyy, xxzz, yyzz;                   // fourth order
};

// Reference state of the stored deviations g = f - f_eq(rho_ref, U), lattice units;
// q[k]: the constant Q_k(j_ref)/rho_ref parts of the equilibrium moments (zero for U = 0).
struct StoreRef3 {
    float rho, jx, jy, jz, ux, uy, uz;
    float qxx, qyy, qzz, qxy, qxz, qyz, qxxyy, qxxzz, qyyzz;
};

struct StepArgs3 {
    int nx, ny, nz;
    Rates3 s;
    StoreRef3 ref;
    float amp_t;         // prescribed mode: A cos(2 pi t / P) / lambda at this step
    const float* ut0;    // prescribed base field [3][n]
};

LBMRV_HD float wgt3(int j) { return j == 0 ? (1.0f / 3.0f) : (j < 7 ? (1.0f / 18.0f) : (1.0f / 36.0f)); }

// Sums of the deviations: drho = sum g, j = sum c g (deviation parts).
struct NodeMoments3 {
    float drho, jx, jy, jz;
};

LBMRV_HD NodeMoments3 node_moments3(const float g[19]) {
    NodeMoments3 m;
    const float xe = (g[7] - g[8]) + (g[9] - g[10]);    // x-y edges, sum cx
    const float ye = (g[7] - g[8]) - (g[9] - g[10]);    // x-y edges, sum cy
    const float xz = (g[11] - g[12]) + (g[13] - g[14]);  // x-z edges, sum cx
    const float zx = (g[11] - g[12]) - (g[13] - g[14]);  // x-z edges, sum cz
    const float yz = (g[15] - g[16]) + (g[17] - g[18]);  // y-z edges, sum cy
    const float zy = (g[15] - g[16]) - (g[17] - g[18]);  // y-z edges, sum cz
    m.drho = (((g[0] + (g[1] + g[2])) + ((g[3] + g[4]) + (g[5] + g[6]))) +
              (((g[7] + g[8]) + (g[9] + g[10])) + ((g[11] + g[12]) + (g[13] + g[14])) +
               ((g[15] + g[16]) + (g[17] + g[18]))));
    m.jx = (g[1] - g[2]) + xe + xz;
    m.jy = (g[3] - g[4]) + ye + yz;
    m.jz = (g[5] - g[6]) + zx + zy;
    return m;
}

// The relaxation at one node, in place on the deviations g, for u = u~ / lambda.
LBMRV_HD void relax_node3(float g[19], float ux, float uy, float uz, const Rates3& s,
                          const StoreRef3& ref) {
    const NodeMoments3 mo = node_moments3(g);
    const float ir = recip(ref.rho + mo.drho);
    const float jx = ref.jx + mo.jx, jy = ref.jy + mo.jy, jz = ref.jz + mo.jz;
    const float jxx = jx * jx * ir, jyy = jy * jy * ir, jzz = jz * jz * ir;
    const float third = 1.0f / 3.0f, ninth = 1.0f / 9.0f;

    // Raw moments of g (deviation part) and d = m(0) - m_eq(0) of the 15 non-conserved
    // monomials. m_eq of the D3Q19 second-order equilibrium: XX: rho/3 + jx^2/rho,
    // XY: jx jy / rho, XY^2: jx/3, X^2Y^2: rho/9 + ((jx^2 + jy^2)/3 - jz^2/6)/rho.
    const float exy = (g[7] + g[8]) + (g[9] + g[10]);
    const float exz = (g[11] + g[12]) + (g[13] + g[14]);
    const float eyz = (g[15] + g[16]) + (g[17] + g[18]);
    const float d_xx = ((g[1] + g[2]) + exy + exz) - third * mo.drho + ref.qxx - jxx;
    const float d_yy = ((g[3] + g[4]) + exy + eyz) - third * mo.drho + ref.qyy - jyy;
    const float d_zz = ((g[5] + g[6]) + exz + eyz) - third * mo.drho + ref.qzz - jzz;
    const float d_xy = ((g[7] + g[8]) - (g[9] + g[10])) + ref.qxy - jx * jy * ir;
    const float d_xz = ((g[11] + g[12]) - (g[13] + g[14])) + ref.qxz - jx * jz * ir;
    const float d_yz = ((g[15] + g[16]) - (g[17] + g[18])) + ref.qyz - jy * jz * ir;
    const float d_xyy = ((g[7] - g[8]) + (g[9] - g[10])) - third * mo.jx;
    const float d_xzz = ((g[11] - g[12]) + (g[13] - g[14])) - third * mo.jx;
    const float d_yxx = ((g[7] - g[8]) - (g[9] - g[10])) - third * mo.jy;
    const float d_yzz = ((g[15] - g[16]) + (g[17] - g[18])) - third * mo.jy;
    const float d_zxx = ((g[11] - g[12]) - (g[13] - g[14])) - third * mo.jz;
    const float d_zyy = ((g[15] - g[16]) - (g[17] - g[18])) - third * mo.jz;
    const float d_xxyy = exy - ninth * mo.drho + ref.qxxyy - (third * (jxx + jyy) - (1.0f / 6.0f) * jzz);
    const float d_xxzz = exz - ninth * mo.drho + ref.qxxzz - (third * (jxx + jzz) - (1.0f / 6.0f) * jyy);
    const float d_yyzz = eyz - ninth * mo.drho + ref.qyyzz - (third * (jyy + jzz) - (1.0f / 6.0f) * jxx);

    // Forward shift T(u~): binomial expansion, lower non-conserved degrees only.
    const float k_xyy = d_xyy - 2.0f * uy * d_xy - ux * d_yy;
    const float k_xzz = d_xzz - 2.0f * uz * d_xz - ux * d_zz;
    const float k_yxx = d_yxx - 2.0f * ux * d_xy - uy * d_xx;
    const float k_yzz = d_yzz - 2.0f * uz * d_yz - uy * d_zz;
    const float k_zxx = d_zxx - 2.0f * ux * d_xz - uz * d_xx;
    const float k_zyy = d_zyy - 2.0f * uy * d_yz - uz * d_yy;
    const float k_xxyy = d_xxyy - 2.0f * uy * d_yxx - 2.0f * ux * d_xyy + uy * uy * d_xx +
                         ux * ux * d_yy + 4.0f * ux * uy * d_xy;
    const float k_xxzz = d_xxzz - 2.0f * uz * d_zxx - 2.0f * ux * d_xzz + uz * uz * d_xx +
                         ux * ux * d_zz + 4.0f * ux * uz * d_xz;
    const float k_yyzz = d_yyzz - 2.0f * uz * d_zyy - 2.0f * uy * d_yzz + uz * uz * d_yy +
                         uy * uy * d_zz + 4.0f * uy * uz * d_yz;

    // Relaxation S, diagonal in the basis polynomials.
    const float tr = d_xx + d_yy + d_zz, da = d_xx - d_yy, db = d_yy - d_zz;
    const float rt = s.e * tr, ra = s.a * da, rb = s.b * db;
    const float r_xx = third * (rt + 2.0f * ra + rb);
    const float r_yy = third * (rt - ra + rb);
    const float r_zz = third * (rt - ra - 2.0f * rb);
    const float r_xy = s.xy * d_xy, r_xz = s.xz * d_xz, r_yz = s.yz * d_yz;
    const float r_xyy = s.xyy * k_xyy, r_xzz = s.xzz * k_xzz, r_yxx = s.yxx * k_yxx;
    const float r_yzz = s.yzz * k_yzz, r_zxx = s.zxx * k_zxx, r_zyy = s.zyy * k_zyy;
    const float r_xxyy = s.xxyy * k_xxyy, r_xxzz = s.xxzz * k_xxzz, r_yyzz = s.yyzz * k_yyzz;

    // Back shift T(-u~) (morphism).
    const float h_xyy = r_xyy + 2.0f * uy * r_xy + ux * r_yy;
    const float h_xzz = r_xzz + 2.0f * uz * r_xz + ux * r_zz;
    const float h_yxx = r_yxx + 2.0f * ux * r_xy + uy * r_xx;
    const float h_yzz = r_yzz + 2.0f * uz * r_yz + uy * r_zz;
    const float h_zxx = r_zxx + 2.0f * ux * r_xz + uz * r_xx;
    const float h_zyy = r_zyy + 2.0f * uy * r_yz + uz * r_yy;
    const float h_xxyy = r_xxyy + 2.0f * uy * r_yxx + 2.0f * ux * r_xyy + uy * uy * r_xx +
                         ux * ux * r_yy + 4.0f * ux * uy * r_xy;
    const float h_xxzz = r_xxzz + 2.0f * uz * r_zxx + 2.0f * ux * r_xzz + uz * uz * r_xx +
                         ux * ux * r_zz + 4.0f * ux * uz * r_xz;
    const float h_yyzz = r_yyzz + 2.0f * uz * r_zyy + 2.0f * uy * r_yzz + uz * uz * r_yy +
                         uy * uy * r_zz + 4.0f * uy * uz * r_yz;

    // f* = f - M(0)^{-1} h, M(0) the monomial moment matrix restricted to zero conserved
    // moments: edges from their four moments, faces from the second-order sums and the
    // momentum balance, rest from the mass balance.
    const float ex1 = 0.5f * (h_xxyy + r_xy), ex2 = 0.5f * (h_xxyy - r_xy);
    const float ox1 = 0.5f * (h_xyy + h_yxx), ox2 = 0.5f * (h_xyy - h_yxx);
    g[7] -= 0.5f * (ex1 + ox1);
    g[8] -= 0.5f * (ex1 - ox1);
    g[9] -= 0.5f * (ex2 + ox2);
    g[10] -= 0.5f * (ex2 - ox2);
    const float ez1 = 0.5f * (h_xxzz + r_xz), ez2 = 0.5f * (h_xxzz - r_xz);
    const float oz1 = 0.5f * (h_xzz + h_zxx), oz2 = 0.5f * (h_xzz - h_zxx);
    g[11] -= 0.5f * (ez1 + oz1);
    g[12] -= 0.5f * (ez1 - oz1);
    g[13] -= 0.5f * (ez2 + oz2);
    g[14] -= 0.5f * (ez2 - oz2);
    const float ey1 = 0.5f * (h_yyzz + r_yz), ey2 = 0.5f * (h_yyzz - r_yz);
    const float oy1 = 0.5f * (h_yzz + h_zyy), oy2 = 0.5f * (h_yzz - h_zyy);
    g[15] -= 0.5f * (ey1 + oy1);
    g[16] -= 0.5f * (ey1 - oy1);
    g[17] -= 0.5f * (ey2 + oy2);
    g[18] -= 0.5f * (ey2 - oy2);
    const float sx = r_xx - h_xxyy - h_xxzz, sy = r_yy - h_xxyy - h_yyzz,
                sz = r_zz - h_xxzz - h_yyzz;
    const float mx = h_xyy + h_xzz, my = h_yxx + h_yzz, mz = h_zxx + h_zyy;
    g[1] -= 0.5f * (sx - mx);
    g[2] -= 0.5f * (sx + mx);
    g[3] -= 0.5f * (sy - my);
    g[4] -= 0.5f * (sy + my);
    g[5] -= 0.5f * (sz - mz);
    g[6] -= 0.5f * (sz + mz);
    g[0] -= (h_xxyy + h_xxzz + h_yyzz) - (r_xx + r_yy + r_zz);
}

}  // namespace lbmrv
