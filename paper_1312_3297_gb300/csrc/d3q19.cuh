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

// The relaxation, in place on the deviations g of one node (R = float) or of two nodes
// (R = F2, one per lane), for u = u~ / lambda. UM = UM_FLUID takes u~ = q / rho of the
// state being relaxed (ux, uy, uz are outputs then); UM = UM_ZERO is the fixed-frame scheme.
// RCP: the form of 1/rho (see recip). INCR = true leaves the increment g* - g in g instead
// of g* (the caller adds it to the input, which it need not keep in registers meanwhile).
template <int UM, int RCP = RCP_RN, bool INCR = false, typename R>
LBMRV_HD void relax_node3(R g[19], R& ux, R& uy, R& uz, const Rates3& s,
                          const StoreRef3& ref) {
    // Sums and differences of opposite populations.
    const R a1 = g[1] + g[2], b1 = g[1] - g[2], a3 = g[3] + g[4], b3 = g[3] - g[4];
    const R a5 = g[5] + g[6], b5 = g[5] - g[6];
    const R a7 = g[7] + g[8], b7 = g[7] - g[8], a9 = g[9] + g[10], b9 = g[9] - g[10];
    const R a11 = g[11] + g[12], b11 = g[11] - g[12], a13 = g[13] + g[14], b13 = g[13] - g[14];
    const R a15 = g[15] + g[16], b15 = g[15] - g[16], a17 = g[17] + g[18], b17 = g[17] - g[18];
    const R exy = a7 + a9, exz = a11 + a13, eyz = a15 + a17;   // edge sums
    const R xe = b7 + b9, ye = b7 - b9;     // x-y edges: sum cx (= X Y^2), sum cy (= Y X^2)
    const R xz = b11 + b13, zx = b11 - b13; // x-z edges: sum cx (= X Z^2), sum cz (= Z X^2)
    const R yz = b15 + b17, zy = b15 - b17; // y-z edges: sum cy (= Y Z^2), sum cz (= Z Y^2)
    // Conserved moments.
    const R drho = (g[0] + ((a1 + a3) + a5)) + ((exy + exz) + eyz);
    const R mjx = b1 + (xe + xz), mjy = b3 + (ye + yz), mjz = b5 + (zx + zy);
    const R ir = recip<RCP>(R(ref.rho) + drho);
    const R jx = R(ref.jx) + mjx, jy = R(ref.jy) + mjy, jz = R(ref.jz) + mjz;
    const R vx = jx * ir, vy = jy * ir, vz = jz * ir;
    if constexpr (UM == UM_FLUID) {
        ux = vx;
        uy = vy;
        uz = vz;
    }
    const R kx = jx * vx, ky = jy * vy, kz = jz * vz;  // jx^2 / rho, ...
    const R third = R(1.0f / 3.0f);

    // d = m(0) - m_eq(0) of the 15 non-conserved monomials. m_eq of the D3Q19 second-order
    // equilibrium: XX: rho/3 + jx^2/rho, XY: jx jy / rho, XY^2: jx/3,
    // X^2Y^2: rho/9 + ((jx^2 + jy^2)/3 - jz^2/6)/rho = rho/9 + |j|^2/(3 rho) - jz^2/(2 rho).
    const R t3 = third * drho;
    const R base = fma_(third, (kx + ky) + kz, R(1.0f / 9.0f) * drho);
    const R d_xx = ((a1 + exy) + exz) - ((t3 + kx) - R(ref.qxx));
    const R d_yy = ((a3 + exy) + eyz) - ((t3 + ky) - R(ref.qyy));
    const R d_zz = ((a5 + exz) + eyz) - ((t3 + kz) - R(ref.qzz));
    const R d_xy = (a7 - a9) - fma_(jx, vy, R(-ref.qxy));
    const R d_xz = (a11 - a13) - fma_(jx, vz, R(-ref.qxz));
    const R d_yz = (a15 - a17) - fma_(jy, vz, R(-ref.qyz));
    const R m3 = R(-1.0f / 3.0f);
    const R d_xyy = fma_(m3, mjx, xe), d_xzz = fma_(m3, mjx, xz);
    const R d_yxx = fma_(m3, mjy, ye), d_yzz = fma_(m3, mjy, yz);
    const R d_zxx = fma_(m3, mjz, zx), d_zyy = fma_(m3, mjz, zy);
    const R d_xxyy = (exy + R(ref.qxxyy)) - fma_(R(-0.5f), kz, base);
    const R d_xxzz = (exz + R(ref.qxxzz)) - fma_(R(-0.5f), ky, base);
    const R d_yyzz = (eyz + R(ref.qyyzz)) - fma_(R(-0.5f), kx, base);

    // Relaxation of the second order, diagonal in (trace, X^2-Y^2, Y^2-Z^2, XY, XZ, YZ).
    const R rt = R(s.e) * ((d_xx + d_yy) + d_zz);
    const R ra = R(s.a) * (d_xx - d_yy), rb = R(s.b) * (d_yy - d_zz);
    const R rtb = rt + rb;
    const R r_xx = third * fma_(R(2.0f), ra, rtb);
    const R r_yy = third * (rtb - ra);
    const R r_zz = third * (rt - fma_(R(2.0f), rb, ra));
    const R r_xy = R(s.xy) * d_xy, r_xz = R(s.xz) * d_xz, r_yz = R(s.yz) * d_yz;

    R h_xyy, h_xzz, h_yxx, h_yzz, h_zxx, h_zyy, h_xxyy, h_xxzz, h_yyzz;
    if constexpr (UM == UM_ZERO) {
        h_xyy = R(s.xyy) * d_xyy;
        h_xzz = R(s.xzz) * d_xzz;
        h_yxx = R(s.yxx) * d_yxx;
        h_yzz = R(s.yzz) * d_yzz;
        h_zxx = R(s.zxx) * d_zxx;
        h_zyy = R(s.zyy) * d_zyy;
        h_xxyy = R(s.xxyy) * d_xxyy;
        h_xxzz = R(s.xxzz) * d_xxzz;
        h_yyzz = R(s.yyzz) * d_yyzz;
    } else {
        const R ux2 = ux + ux, uy2 = uy + uy, uz2 = uz + uz;
        const R uxx = ux * ux, uyy = uy * uy, uzz = uz * uz;
        const R uxy4 = ux2 * uy2, uxz4 = ux2 * uz2, uyz4 = uy2 * uz2;
        // Forward shift T(u~): binomial expansion of (X - ux)^a (Y - uy)^b (Z - uz)^c,
        // lower non-conserved degrees only.
        const R k_xyy = d_xyy - fma_(uy2, d_xy, ux * d_yy);
        const R k_xzz = d_xzz - fma_(uz2, d_xz, ux * d_zz);
        const R k_yxx = d_yxx - fma_(ux2, d_xy, uy * d_xx);
        const R k_yzz = d_yzz - fma_(uz2, d_yz, uy * d_zz);
        const R k_zxx = d_zxx - fma_(ux2, d_xz, uz * d_xx);
        const R k_zyy = d_zyy - fma_(uy2, d_yz, uz * d_yy);
        const R k_xxyy = fma_(uyy, d_xx, fma_(uxx, d_yy, fma_(uxy4, d_xy, d_xxyy))) -
                         fma_(uy2, d_yxx, ux2 * d_xyy);
        const R k_xxzz = fma_(uzz, d_xx, fma_(uxx, d_zz, fma_(uxz4, d_xz, d_xxzz))) -
                         fma_(uz2, d_zxx, ux2 * d_xzz);
        const R k_yyzz = fma_(uzz, d_yy, fma_(uyy, d_zz, fma_(uyz4, d_yz, d_yyzz))) -
                         fma_(uz2, d_zyy, uy2 * d_yzz);
        // Relaxation S of the third and fourth orders.
        const R r_xyy = R(s.xyy) * k_xyy, r_xzz = R(s.xzz) * k_xzz, r_yxx = R(s.yxx) * k_yxx;
        const R r_yzz = R(s.yzz) * k_yzz, r_zxx = R(s.zxx) * k_zxx, r_zyy = R(s.zyy) * k_zyy;
        const R r_xxyy = R(s.xxyy) * k_xxyy, r_xxzz = R(s.xxzz) * k_xxzz;
        const R r_yyzz = R(s.yyzz) * k_yyzz;
        // Back shift T(-u~) (morphism).
        h_xyy = fma_(uy2, r_xy, fma_(ux, r_yy, r_xyy));
        h_xzz = fma_(uz2, r_xz, fma_(ux, r_zz, r_xzz));
        h_yxx = fma_(ux2, r_xy, fma_(uy, r_xx, r_yxx));
        h_yzz = fma_(uz2, r_yz, fma_(uy, r_zz, r_yzz));
        h_zxx = fma_(ux2, r_xz, fma_(uz, r_xx, r_zxx));
        h_zyy = fma_(uy2, r_yz, fma_(uz, r_yy, r_zyy));
        h_xxyy = fma_(uy2, r_yxx, fma_(ux2, r_xyy,
                 fma_(uyy, r_xx, fma_(uxx, r_yy, fma_(uxy4, r_xy, r_xxyy)))));
        h_xxzz = fma_(uz2, r_zxx, fma_(ux2, r_xzz,
                 fma_(uzz, r_xx, fma_(uxx, r_zz, fma_(uxz4, r_xz, r_xxzz)))));
        h_yyzz = fma_(uz2, r_zyy, fma_(uy2, r_yzz,
                 fma_(uzz, r_yy, fma_(uyy, r_zz, fma_(uyz4, r_yz, r_yyzz)))));
    }

    // f* = f - M(0)^{-1} h, M(0) the monomial moment matrix restricted to zero conserved
    // moments: edges from their four moments, faces from the second-order sums and the
    // momentum balance, rest from the mass balance.
    const R q4 = R(-0.25f), q2 = R(-0.5f);
    {
        const R p = h_xxyy + r_xy, q = h_xxyy - r_xy, o1 = h_xyy + h_yxx, o2 = h_xyy - h_yxx;
        g[7] = INCR ? q4 * (p + o1) : fma_(q4, p + o1, g[7]);
        g[8] = INCR ? q4 * (p - o1) : fma_(q4, p - o1, g[8]);
        g[9] = INCR ? q4 * (q + o2) : fma_(q4, q + o2, g[9]);
        g[10] = INCR ? q4 * (q - o2) : fma_(q4, q - o2, g[10]);
    }
    {
        const R p = h_xxzz + r_xz, q = h_xxzz - r_xz, o1 = h_xzz + h_zxx, o2 = h_xzz - h_zxx;
        g[11] = INCR ? q4 * (p + o1) : fma_(q4, p + o1, g[11]);
        g[12] = INCR ? q4 * (p - o1) : fma_(q4, p - o1, g[12]);
        g[13] = INCR ? q4 * (q + o2) : fma_(q4, q + o2, g[13]);
        g[14] = INCR ? q4 * (q - o2) : fma_(q4, q - o2, g[14]);
    }
    {
        const R p = h_yyzz + r_yz, q = h_yyzz - r_yz, o1 = h_yzz + h_zyy, o2 = h_yzz - h_zyy;
        g[15] = INCR ? q4 * (p + o1) : fma_(q4, p + o1, g[15]);
        g[16] = INCR ? q4 * (p - o1) : fma_(q4, p - o1, g[16]);
        g[17] = INCR ? q4 * (q + o2) : fma_(q4, q + o2, g[17]);
        g[18] = INCR ? q4 * (q - o2) : fma_(q4, q - o2, g[18]);
    }
    const R sx = r_xx - (h_xxyy + h_xxzz), sy = r_yy - (h_xxyy + h_yyzz);
    const R sz = r_zz - (h_xxzz + h_yyzz);
    const R mx = h_xyy + h_xzz, my = h_yxx + h_yzz, mz = h_zxx + h_zyy;
    g[1] = INCR ? q2 * (sx - mx) : fma_(q2, sx - mx, g[1]);
    g[2] = INCR ? q2 * (sx + mx) : fma_(q2, sx + mx, g[2]);
    g[3] = INCR ? q2 * (sy - my) : fma_(q2, sy - my, g[3]);
    g[4] = INCR ? q2 * (sy + my) : fma_(q2, sy + my, g[4]);
    g[5] = INCR ? q2 * (sz - mz) : fma_(q2, sz - mz, g[5]);
    g[6] = INCR ? q2 * (sz + mz) : fma_(q2, sz + mz, g[6]);
    g[0] = INCR ? rt - ((h_xxyy + h_xxzz) + h_yyzz) : g[0] - (((h_xxyy + h_xxzz) + h_yyzz) - rt);
}

}  // namespace lbmrv
