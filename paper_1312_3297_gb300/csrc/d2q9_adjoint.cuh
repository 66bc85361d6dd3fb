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

// The reverse relaxation of one node (R = F1, scalar FP32 whose arithmetic the compiler does
// not contract) or of two nodes at once (R = F2, one node per lane, packed FP32
// instructions). Every fused multiply-add is written out.
// UM = UM_FLUID takes u = q / rho of the node (ux, uy are ignored) and folds dL/du into the
// moments' adjoint; UM = UM_ZERO is the fixed-frame scheme. RCP: the form of 1/rho (see
// recip).
//   g      the pre-relaxation deviations (as pulled by the forward step)
//   a      dL/dg*, the adjoint of the relaxed deviations
//   out    dL/dg = a^T dg*/dg
//   sbar   += dL/ds for (e, p_xx, p_xy, q_x, q_y, eps)
//   uxbar, uybar  a^T dg*/du (0 for UM_ZERO and UM_FLUID)
template <int UM, int RCP, typename R>
LBMRV_HD void relax_node_vjp(const R g[9], const R a[9], R ux, R uy, const Rates& s,
                             const StoreRef& ref, R out[9], R sbar[6], R& uxbar, R& uybar) {
    // ---- forward recompute: the relations of relax_node
    const R a1 = g[1] + g[3], b1 = g[1] - g[3], a2 = g[2] + g[4], b2 = g[2] - g[4];
    const R a5 = g[5] + g[7], b5 = g[5] - g[7], a6 = g[6] + g[8], b6 = g[6] - g[8];
    const R s1 = a1 + a2, s2 = a5 + a6, bm = b5 - b6, bp = b5 + b6;
    const R drho = g[0] + (s1 + s2);
    const R ir = recip<RCP>(R(ref.rho) + drho);
    const R jx = R(ref.jx) + (b1 + bm), jy = R(ref.jy) + (b2 + bp);
    const R vx = jx * ir, vy = jy * ir;  // q / (rho lambda)
    if constexpr (UM == UM_FLUID) {
        ux = vx;
        uy = vy;
    }
    const R kx = jx * vx, ky = jy * vy;
    const R kin = kx + ky, kxy = kx - ky;  // |j|^2 / rho, (jx^2 - jy^2) / rho
    const R d_e = fma_(R(4.0f), s2, fma_(R(-2.0f), g[0], s1)) - fma_(R(3.0f), kin, R(-ref.c[0]));
    const R d_xx = (a1 - a2) - (kxy - R(ref.c[1]));
    const R d_xy = (a5 - a6) - fma_(jx, vy, R(-ref.c[2]));
    const R d_qx = (bm + bm) - b1;
    const R d_qy = (bp + bp) - b2;
    const R d_ep = fma_(R(3.0f), g[0] - s1, fma_(R(3.0f), kin, R(ref.c[5])));

    R ux2, uy2, ux3, uy3, ux6, uy6, d3e, d3xx, d3xy;
    R t_qx = d_qx, t_qy = d_qy, t_ep = d_ep;  // t = T6(u) d (identity for u = 0)
    if constexpr (UM != UM_ZERO) {
        ux2 = ux + ux;
        uy2 = uy + uy;
        ux3 = ux2 + ux;
        uy3 = uy2 + uy;
        ux6 = ux3 + ux3;
        uy6 = uy3 + uy3;
        d3e = fma_(ux6, ux, uy6 * uy);  // 6 |u|^2
        d3xx = ux3 * ux3 - uy3 * uy3;   // 9 (ux^2 - uy^2)
        d3xy = ux6 * uy6;               // 36 ux uy
        t_qx = d_qx - fma_(ux2, d_e, fma_(ux3, d_xx, uy6 * d_xy));
        t_qy = fma_(uy3, d_xx, d_qy) - fma_(uy2, d_e, ux6 * d_xy);
        t_ep = fma_(d3e, d_e, fma_(d3xx, d_xx, fma_(d3xy, d_xy, d_ep))) -
               fma_(ux6, d_qx, uy6 * d_qy);
    }

    // ---- reverse. g* = g - M(0)^T diag(1/|row|^2) h: hb = dL/dh = -diag(1/|row|^2) M(0) a
    // on (e, p_xx, p_xy, q_x, q_y, eps), |row|^2 = 36, 4, 4, 12, 12, 36.
    const R aa1 = a[1] + a[3], ab1 = a[1] - a[3], aa2 = a[2] + a[4], ab2 = a[2] - a[4];
    const R aa5 = a[5] + a[7], ab5 = a[5] - a[7], aa6 = a[6] + a[8], ab6 = a[6] - a[8];
    const R sa1 = aa1 + aa2, sa2 = aa5 + aa6, abm = ab5 - ab6, abp = ab5 + ab6;
    const R hb_e = fma_(R(4.0f), a[0], fma_(R(-2.0f), sa2, sa1)) * R(1.0f / 36.0f);
    const R hb_xx = (aa2 - aa1) * R(0.25f);
    const R hb_xy = (aa6 - aa5) * R(0.25f);
    const R hb_qx = ((ab1 + ab1) - abm) * R(1.0f / 12.0f);
    const R hb_qy = ((ab2 + ab2) - abp) * R(1.0f / 12.0f);
    const R hb_ep = fma_(R(-4.0f), a[0], (sa1 + sa1) - sa2) * R(1.0f / 36.0f);

    // h = T6(-u) r  ->  rb = T6(-u)^T hb
    R rb_e = hb_e, rb_xx = hb_xx, rb_xy = hb_xy, rb_qx = hb_qx, rb_qy = hb_qy;
    const R rb_ep = hb_ep;
    if constexpr (UM != UM_ZERO) {
        rb_qx = fma_(ux6, hb_ep, hb_qx);
        rb_qy = fma_(uy6, hb_ep, hb_qy);
        rb_e = fma_(ux2, hb_qx, fma_(uy2, hb_qy, fma_(d3e, hb_ep, hb_e)));
        rb_xx = fma_(ux3, hb_qx, fma_(d3xx, hb_ep, hb_xx)) - uy3 * hb_qy;
        rb_xy = fma_(uy6, hb_qx, fma_(ux6, hb_qy, fma_(d3xy, hb_ep, hb_xy)));
    }

    // r = S t: the rate gradients, and tb = S rb
    sbar[0] = fma_(rb_e, d_e, sbar[0]);
    sbar[1] = fma_(rb_xx, d_xx, sbar[1]);
    sbar[2] = fma_(rb_xy, d_xy, sbar[2]);
    sbar[3] = fma_(rb_qx, t_qx, sbar[3]);
    sbar[4] = fma_(rb_qy, t_qy, sbar[4]);
    sbar[5] = fma_(rb_ep, t_ep, sbar[5]);
    const R tb_e = R(s.e) * rb_e, tb_xx = R(s.pxx) * rb_xx, tb_xy = R(s.pxy) * rb_xy;
    const R tb_qx = R(s.qx) * rb_qx, tb_qy = R(s.qy) * rb_qy, tb_ep = R(s.eps) * rb_ep;

    // t = T6(u) d  ->  db = T6(u)^T tb, and the adjoint of u through both shifts
    R db_e = tb_e, db_xx = tb_xx, db_xy = tb_xy, db_qx = tb_qx, db_qy = tb_qy;
    const R db_ep = tb_ep;
    R ubx = R(0.0f), uby = R(0.0f);
    if constexpr (UM != UM_ZERO) {
        db_qx = tb_qx - ux6 * tb_ep;
        db_qy = tb_qy - uy6 * tb_ep;
        db_e = fma_(d3e, tb_ep, tb_e) - fma_(ux2, tb_qx, uy2 * tb_qy);
        db_xx = fma_(uy3, tb_qy, fma_(d3xx, tb_ep, tb_xx)) - ux3 * tb_qx;
        db_xy = fma_(d3xy, tb_ep, tb_xy) - fma_(uy6, tb_qx, ux6 * tb_qy);
        // r = S t with t = T6(u) d and h = T6(-u) r, differentiated in u:
        //   ubx = hb_qx (2 r_e + 3 r_xx) - tb_qx (2 d_e + 3 d_xx) + 6 (hb_qy r_xy - tb_qy d_xy)
        //       + 6 (hb_ep r_qx - tb_ep d_qx) + 6ux (2 P_e + 3 P_xx) + 6uy (6 P_xy),
        //   uby = hb_qy (2 r_e - 3 r_xx) - tb_qy (2 d_e - 3 d_xx) + 6 (hb_qx r_xy - tb_qx d_xy)
        //       + 6 (hb_ep r_qy - tb_ep d_qy) + 6uy (2 P_e - 3 P_xx) + 6ux (6 P_xy),
        // with P_k = hb_ep r_k + tb_ep d_k (the u-dependence of the eps rows).
        const R r_e = R(s.e) * d_e, r_xx = R(s.pxx) * d_xx, r_xy = R(s.pxy) * d_xy;
        const R r_qx = R(s.qx) * t_qx, r_qy = R(s.qy) * t_qy;
        const R p_e = fma_(hb_ep, r_e, tb_ep * d_e);
        const R p_xx = fma_(hb_ep, r_xx, tb_ep * d_xx);
        const R p_xy = fma_(hb_ep, r_xy, tb_ep * d_xy);
        const R re2 = r_e + r_e, rx3 = R(3.0f) * r_xx;
        const R de2 = d_e + d_e, dx3 = R(3.0f) * d_xx;
        const R pe2 = p_e + p_e, px3 = R(3.0f) * p_xx, pxy6 = R(6.0f) * p_xy;
        const R wx = fma_(hb_qy, r_xy, hb_ep * r_qx) - fma_(tb_qy, d_xy, tb_ep * d_qx);
        const R wy = fma_(hb_qx, r_xy, hb_ep * r_qy) - fma_(tb_qx, d_xy, tb_ep * d_qy);
        ubx = fma_(hb_qx, re2 + rx3, fma_(ux6, pe2 + px3, fma_(uy6, pxy6, R(6.0f) * wx))) -
              tb_qx * (de2 + dx3);
        uby = fma_(hb_qy, re2 - rx3, fma_(uy6, pe2 - px3, fma_(ux6, pxy6, R(6.0f) * wy))) -
              tb_qy * (de2 - dx3);
    }

    // d = M(0) g - m_eq(0)(rho, j) + const: rho enters through 2 drho (e) and -drho (eps),
    // j through the q rows and the quadratic terms kin = |j|^2/rho (-3 in e, +3 in eps),
    // kxy = (jx^2 - jy^2)/rho (-1 in p_xx), jx jy / rho (-1 in p_xy).
    const R kinb = R(3.0f) * (db_ep - db_e);
    R jxb = fma_(vx + vx, kinb - db_xx, db_qx) - vy * db_xy;
    R jyb = fma_(vy + vy, kinb + db_xx, db_qy) - vx * db_xy;
    const R vxx = vx * vx, vyy = vy * vy;
    R drhob = ((db_e + db_e) - db_ep) -
              (fma_(vxx + vyy, kinb, (vyy - vxx) * db_xx) - (vx * vy) * db_xy);
    if constexpr (UM == UM_FLUID) {  // u = j / rho
        jxb = fma_(ir, ubx, jxb);
        jyb = fma_(ir, uby, jyb);
        drhob = drhob - ir * fma_(vx, ubx, vy * uby);
        ubx = R(0.0f);
        uby = R(0.0f);
    }

    // out = a + M(0)^T db (non-conserved rows) + drhob + c . jb
    const R axis = drhob - (db_e + (db_ep + db_ep));
    const R diag = drhob + ((db_e + db_e) + db_ep);
    const R x1 = jxb - (db_qx + db_qx), y1 = jyb - (db_qy + db_qy);
    const R x2 = db_qx + jxb, y2 = db_qy + jyb;
    const R pp = x2 + y2, pm = y2 - x2;
    const R ax_p = axis + db_xx, ax_m = axis - db_xx;
    const R dg_p = diag + db_xy, dg_m = diag - db_xy;
    out[0] = a[0] + fma_(R(4.0f), db_ep - db_e, drhob);
    out[1] = a[1] + (ax_p + x1);
    out[3] = a[3] + (ax_p - x1);
    out[2] = a[2] + (ax_m + y1);
    out[4] = a[4] + (ax_m - y1);
    out[5] = a[5] + (dg_p + pp);
    out[7] = a[7] + (dg_p - pp);
    out[6] = a[6] + (dg_m + pm);
    out[8] = a[8] + (dg_m - pm);
    uxbar = ubx;
    uybar = uby;
}

}  // namespace lbmrv
