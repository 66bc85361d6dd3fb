// Discrete adjoint of the D2Q9 relative-velocity relaxation: the transposed Jacobian of
// relax_node (d2q9.cuh) applied to an adjoint vector, node by node.
//
// Forward (per node, deviations g, u = u~/lambda):
//   rho = rho_ref + sum g, j = j_ref + sum c g, d = m(0) - m_eq(0) on the six non-conserved
//   moments, t = T6(u) d, r = S t, h = T6(-u) r, g* = g - M(0)^{-1} h.
// The reverse sweep below walks these relations backwards (hand-derived), recomputing the
// forward intermediates in registers. It returns a^T dg*/dg, the per-node contributions to
// dL/ds_k for the six non-conserved rates, and a^T dg*/du (used for a prescribed u~;
// for u~ = q/rho it is folded into the moments' adjoint).
#pragma once

#include "d2q9.cuh"

namespace lbmrv {

// out_j = sum_k M(0)_kj v_k over the six non-conserved moments (E, XX, XY, QX, QY, EP).
LBMRV_HD void mT6(float E, float XX, float XY, float QX, float QY, float EP,
                                    float out[9]) {
    const float axis_c = -E - 2.0f * EP, diag_c = 2.0f * E + EP;
    out[0] = -4.0f * E + 4.0f * EP;
    out[1] = axis_c + XX - 2.0f * QX;
    out[2] = axis_c - XX - 2.0f * QY;
    out[3] = axis_c + XX + 2.0f * QX;
    out[4] = axis_c - XX + 2.0f * QY;
    out[5] = diag_c + XY + QX + QY;
    out[6] = diag_c - XY - QX + QY;
    out[7] = diag_c + XY - QX - QY;
    out[8] = diag_c - XY + QX - QY;
}

template <int UM>
LBMRV_HD void relax_node_vjp(const float g[9], const float a[9], float ux,
                                               float uy, const Rates& s, const StoreRef& ref,
                                               float out[9], float sbar[6], float& uxbar,
                                               float& uybar) {
    // ---- forward recompute
    const NodeMoments mo = node_moments(g);
    const float ir = recip(ref.rho + mo.drho);
    const float jx = ref.jx + mo.jx, jy = ref.jy + mo.jy;
    const float jxx = jx * jx * ir, jyy = jy * jy * ir, pxye = jx * jy * ir;
    const float jj3 = 3.0f * (jxx + jyy);
    const float s1 = (g[1] + g[2]) + (g[3] + g[4]);
    const float s2 = (g[5] + g[6]) + (g[7] + g[8]);
    const float ga = g[5] - g[7], gb = g[6] - g[8];
    const float d_e = (-4.0f * g[0] - s1 + 2.0f * s2) + ref.c[0] + 2.0f * mo.drho - jj3;
    const float d_xx = ((g[1] + g[3]) - (g[2] + g[4])) + ref.c[1] - (jxx - jyy);
    const float d_xy = ((g[5] + g[7]) - (g[6] + g[8])) + ref.c[2] - pxye;
    const float d_qx = (-2.0f * (g[1] - g[3]) + (ga - gb)) + ref.c[3] + jx;
    const float d_qy = (-2.0f * (g[2] - g[4]) + (ga + gb)) + ref.c[4] + jy;
    const float d_ep = (4.0f * g[0] - 2.0f * s1 + s2) + ref.c[5] - mo.drho + jj3;
    const float ux2 = ux * ux, uy2 = uy * uy, uxy = ux * uy;
    const float d3e = 6.0f * (ux2 + uy2), d3xx = 9.0f * (ux2 - uy2), d3xy = 36.0f * uxy;
    const float t_qx = d_qx - 2.0f * ux * d_e - 3.0f * ux * d_xx - 6.0f * uy * d_xy;
    const float t_qy = d_qy - 2.0f * uy * d_e + 3.0f * uy * d_xx - 6.0f * ux * d_xy;
    const float t_ep = d_ep + d3e * d_e + d3xx * d_xx + d3xy * d_xy - 6.0f * ux * d_qx -
                       6.0f * uy * d_qy;
    const float r_e = s.e * d_e, r_xx = s.pxx * d_xx, r_xy = s.pxy * d_xy;
    const float r_qx = s.qx * t_qx, r_qy = s.qy * t_qy;

    // ---- reverse: g* = g - M(0)^{-1} h  ->  cbar = -M(0) a, then the 1/|row|^2 scaling
    const float sa1 = (a[1] + a[2]) + (a[3] + a[4]);
    const float sa2 = (a[5] + a[6]) + (a[7] + a[8]);
    const float aa = a[5] - a[7], ab = a[6] - a[8];
    const float rb_e0 = (4.0f * a[0] + sa1 - 2.0f * sa2) * (1.0f / 36.0f);
    const float rb_xx0 = -((a[1] + a[3]) - (a[2] + a[4])) * 0.25f;
    const float rb_xy0 = -((a[5] + a[7]) - (a[6] + a[8])) * 0.25f;
    const float hb_qx = (2.0f * (a[1] - a[3]) - (aa - ab)) * (1.0f / 12.0f);
    const float hb_qy = (2.0f * (a[2] - a[4]) - (aa + ab)) * (1.0f / 12.0f);
    const float hb_ep = -(4.0f * a[0] - 2.0f * sa1 + sa2) * (1.0f / 36.0f);

    // h = T6(-u) r
    const float rb_qx = hb_qx + 6.0f * ux * hb_ep;
    const float rb_qy = hb_qy + 6.0f * uy * hb_ep;
    const float rb_ep = hb_ep;
    const float rb_e = rb_e0 + 2.0f * ux * hb_qx + 2.0f * uy * hb_qy + d3e * hb_ep;
    const float rb_xx = rb_xx0 + 3.0f * ux * hb_qx - 3.0f * uy * hb_qy + d3xx * hb_ep;
    const float rb_xy = rb_xy0 + 6.0f * uy * hb_qx + 6.0f * ux * hb_qy + d3xy * hb_ep;

    // r = S t (rates), and their gradients
    const float db_e0 = s.e * rb_e, db_xx0 = s.pxx * rb_xx, db_xy0 = s.pxy * rb_xy;
    const float tb_qx = s.qx * rb_qx, tb_qy = s.qy * rb_qy, tb_ep = s.eps * rb_ep;
    sbar[0] += rb_e * d_e;
    sbar[1] += rb_xx * d_xx;
    sbar[2] += rb_xy * d_xy;
    sbar[3] += rb_qx * t_qx;
    sbar[4] += rb_qy * t_qy;
    sbar[5] += rb_ep * t_ep;

    // t = T6(u) d
    const float db_qx = tb_qx - 6.0f * ux * tb_ep;
    const float db_qy = tb_qy - 6.0f * uy * tb_ep;
    const float db_ep = tb_ep;
    const float db_e = db_e0 - 2.0f * ux * tb_qx - 2.0f * uy * tb_qy + d3e * tb_ep;
    const float db_xx = db_xx0 - 3.0f * ux * tb_qx + 3.0f * uy * tb_qy + d3xx * tb_ep;
    const float db_xy = db_xy0 - 6.0f * uy * tb_qx - 6.0f * ux * tb_qy + d3xy * tb_ep;

    // adjoint of u through both shifts (zero mode: u is the constant 0)
    float ubx = 0.0f, uby = 0.0f;
    if (UM != UM_ZERO) {
        const float d3eb = hb_ep * r_e + tb_ep * d_e;
        const float d3xxb = hb_ep * r_xx + tb_ep * d_xx;
        const float d3xyb = hb_ep * r_xy + tb_ep * d_xy;
        ubx = hb_qx * (2.0f * r_e + 3.0f * r_xx) + 6.0f * hb_qy * r_xy + 6.0f * hb_ep * r_qx -
              tb_qx * (2.0f * d_e + 3.0f * d_xx) - 6.0f * tb_qy * d_xy - 6.0f * tb_ep * d_qx +
              12.0f * ux * d3eb + 18.0f * ux * d3xxb + 36.0f * uy * d3xyb;
        uby = 6.0f * hb_qx * r_xy + hb_qy * (2.0f * r_e - 3.0f * r_xx) + 6.0f * hb_ep * r_qy -
              6.0f * tb_qx * d_xy + tb_qy * (-2.0f * d_e + 3.0f * d_xx) - 6.0f * tb_ep * d_qy +
              12.0f * uy * d3eb - 18.0f * uy * d3xxb + 36.0f * ux * d3xyb;
    }

    // d = m(0) - m_eq(0)(rho, j)
    float drhob = 2.0f * db_e - db_ep;
    float jxb = db_qx, jyb = db_qy;
    const float jj3b = db_ep - db_e;
    const float jxxb = -db_xx + 3.0f * jj3b, jyyb = db_xx + 3.0f * jj3b, pxyb = -db_xy;
    jxb += 2.0f * jx * ir * jxxb + jy * ir * pxyb;
    jyb += 2.0f * jy * ir * jyyb + jx * ir * pxyb;
    float irb = jx * jx * jxxb + jy * jy * jyyb + jx * jy * pxyb;
    if (UM == UM_FLUID) {  // u = j / rho
        jxb += ir * ubx;
        jyb += ir * uby;
        irb += jx * ubx + jy * uby;
        ubx = 0.0f;
        uby = 0.0f;
    }
    drhob -= ir * ir * irb;

    float mt[9];
    mT6(db_e, db_xx, db_xy, db_qx, db_qy, db_ep, mt);
    out[0] = a[0] + mt[0] + drhob;
    out[1] = a[1] + mt[1] + drhob + jxb;
    out[2] = a[2] + mt[2] + drhob + jyb;
    out[3] = a[3] + mt[3] + drhob - jxb;
    out[4] = a[4] + mt[4] + drhob - jyb;
    out[5] = a[5] + mt[5] + drhob + jxb + jyb;
    out[6] = a[6] + mt[6] + drhob - jxb + jyb;
    out[7] = a[7] + mt[7] + drhob - jxb - jyb;
    out[8] = a[8] + mt[8] + drhob + jxb - jyb;
    uxbar = ubx;
    uybar = uby;
}

}  // namespace lbmrv
