// Per-node LW-ACM update (moment form, see lwacm_core.cuh) shared by the generic
// and the batched kernels.
#pragma once

#include "lwacm_core.cuh"

namespace lwacm {

// Full update of one node (x,y,z). With WALLS, sources beyond a walled face are
// replaced by the bounce-back rule; without, every axis wraps (periodic).
// With NUP the density sums its link values with s_p = 18 nu_p in place of s
// (omega_p of Section 2.2, item 3: only the pressure update changes). With SC a
// passive scalar T (the field after the flow fields) is advanced by Eq. ACM2.0t
// with the velocity at time t:
//   T+(x) = a_t T(x) + sum_i w_i [(1 - a_t)(T + 9/2 e^2 - 3/2 |u|^2) + 3 T e](x - c_i),
// the own node's even parts summing to a_t T(x) (sum_i w_i (9/2 e^2 - 3/2 |u|^2) = 0).
// With BULK (D2Q9, periodic) the source's equilibrium is f^(e*) of Appendix
// "Computing derivatives locally" (Eq. quasi-equilibrium2): f^(e) plus the change of
// the product-form quasi-equilibrium (Eqs. d2q9_equilibrium_gen, quasi-equilibrium)
// when its trace moves from Tr^(e) = 2/3 + |u|^2 to Tr^(e) + gamma (Tr^(+) - Tr^(e)),
// Tr^(+) the trace of the source's last update, stored as the deviation
// Tr^(+) - Tr^(e) (like d = rho - 1: no O(1) constant in single precision). Per
// link the increment is
//   Df = rho [h (ax B + ay A) + ax ay h^2],  h = gamma (Tr^(+) - Tr^(e)) / 2,
// with A = 1 - Pxx (c_x = 0) or (Pxx + c_x u)/2, ax = -1 or 1/2 (B, ay likewise in
// y), Pxx = 1/3 + u^2, Pyy = 1/3 + v^2; it is pre-combined like f^(e), Df - a Df^o,
// with its odd part Df^o = rho h (ax c_y v/2 + ay c_x u/2). The post-combine term
// adds nothing to the trace and sum_i (|c_i|^2 - 2/3) w_i = 0, so
// Tr^(+) - Tr^(e) = sum_i (|c_i|^2 - 2/3) g_i / rho_a - |u+|^2, rho_a the zeroth
// moment of the updated distribution (the new density unless NUP). With NUP as
// well the density pre-combines the increment with a_p: (a - a_p) sum_i Df^o_i =
// (sdelta/3) sum_i Df^o_i more; the momentum and the trace keep a.
template <int Q, bool WALLS, bool NUP = false, bool SC = false, bool BULK = false, typename T>
__device__ __forceinline__ void node_update(const T *__restrict__ in, T *__restrict__ out,
                                            const StepParams &p, int x, int y, int z) {
    using L = Lat<Q>;
    const long long k = ((long long)z * p.ny + y) * p.nx + x;
    const T *Din = in, *Uin = in + p.fstride, *Vin = in + 2 * p.fstride,
            *Win = in + 3 * p.fstride;
    const float dx = ldf(Din + k), ux = ldf(Uin + k), uy = ldf(Vin + k);
    const float uz = (Q == 19) ? ldf(Win + k) : 0.f;
    const float rx = 1.f + dx;
    const float qx = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
    float dd = 0.f, jx = 0.f, jy = 0.f, jz = 0.f, dsp = 0.f, ts = 0.f, trs = 0.f, dfos = 0.f;
    const T *Tin = in + (Q == 19 ? 4 : 3) * p.fstride;
    const float omt = 1.f - p.at;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = L::c(i, 0), cy = L::c(i, 1), cz = L::c(i, 2);
        int sx = x - cx, sy = y - cy, sz = z - cz;
        bool outside = false, above = false;
        if (WALLS) {
            if (p.walled[0] && (sx < 0 || sx >= p.nx)) outside = true;
            if (p.walled[1] && (sy < 0 || sy >= p.ny)) outside = true;
            if (Q == 19 && p.walled[2] && (sz < 0 || sz >= p.nz)) outside = true;
            const int sl = p.lid_axis == 0 ? sx : (p.lid_axis == 1 ? sy : sz);
            const int nl = p.lid_axis == 0 ? p.nx : (p.lid_axis == 1 ? p.ny : p.nz);
            above = outside && sl >= nl;
        }
        // a source beyond a wall reads the node itself (already loaded, its values go
        // unused): no link's loads wait behind the wall test
        sx = sx < 0 ? sx + p.nx : (sx >= p.nx ? sx - p.nx : sx);
        sy = sy < 0 ? sy + p.ny : (sy >= p.ny ? sy - p.ny : sy);
        sz = sz < 0 ? sz + p.nz : (sz >= p.nz ? sz - p.nz : sz);
        const long long s = outside ? k : ((long long)sz * p.ny + sy) * p.nx + sx;
        const float ds = ldf(Din + s), us = ldf(Uin + s), vs = ldf(Vin + s);
        const float ws = (Q == 19) ? ldf(Win + s) : 0.f;
        float g;
        if (!outside) {
            const float e = cx * us + cy * vs + cz * ws;
            const float q = fmaf(us, us, fmaf(vs, vs, ws * ws));
            g = link_g(L::w(i), ds, 1.f + ds, e, q, p.s);
            if (NUP) dsp = fmaf(L::w(i) * (1.f + ds), e, dsp);  // sum of w rho e
            if (SC) {
                const float tsrc = ldf(Tin + s);
                const float even = tsrc + fmaf(4.5f * e, e, -1.5f * q);
                ts = fmaf(L::w(i), fmaf(omt, even, 3.f * tsrc * e), ts);
            }
            if (BULK) {
                const float pxx = fmaf(us, us, 1.f / 3.f), pyy = fmaf(vs, vs, 1.f / 3.f);
                const float h = 0.5f * p.gamma * ldf(Tin + s);
                const float A = cx == 0 ? 1.f - pxx : 0.5f * fmaf((float)cx, us, pxx);
                const float B = cy == 0 ? 1.f - pyy : 0.5f * fmaf((float)cy, vs, pyy);
                const float ax = cx == 0 ? -1.f : 0.5f, ay = cy == 0 ? -1.f : 0.5f;
                const float rs = 1.f + ds;
                const float df = rs * h * fmaf(ax * ay, h, fmaf(ax, B, ay * A));
                const float dfo = rs * h * (0.5f * fmaf(ax * cy, vs, ay * cx * us));
                g += fmaf(-p.a, dfo, df);
                if (NUP) dfos += dfo;
            }
        } else {
            // Eq. ACM2.0cccbb2 + Eq. ACM2.0ccccbb: own outgoing BB(i) value, reflected
            const float e = -(cx * ux + cy * uy + cz * uz);
            g = link_g(L::w(i), dx, rx, e, qx, p.s);
            if (above) {
                const float cu = cx * p.lid[0] + cy * p.lid[1] + cz * p.lid[2];
                g = fmaf(L::w(i) * p.wallc, cu, g);
            }
        }
        dd += g;
        if (BULK) trs = fmaf((float)(cx * cx + cy * cy) - 2.f / 3.f, g, trs);
        if (cx) jx += cx > 0 ? g : -g;
        if (cy) jy += cy > 0 ? g : -g;
        if (cz) jz += cz > 0 ? g : -g;
    }
    const float rna = 1.f + dd;  // zeroth moment of the distribution built with a
    if (NUP) dd = fmaf(p.sdelta, dsp, dd);
    if (NUP && BULK) dd = fmaf(p.sdelta * (1.f / 3.f), dfos, dd);
    const float mx = post_factor(p.a, dx, p.am1);  // a rho u = u + mx u (post_combine)
    jx = post_combine(jx, mx, ux);
    jy = post_combine(jy, mx, uy);
    jz = post_combine(jz, mx, uz);
    if (p.has_force) {  // Eq. force: the odd part of f^(e)(rho(x,t), g) adds rho g to j
        jx = fmaf(rx, p.force[0], jx);
        jy = fmaf(rx, p.force[1], jy);
        jz = fmaf(rx, p.force[2], jz);
    }
    if (p.gfield) {  // Eq. force with a space-dependent g(x,t), supplied per step
        jx = fmaf(rx, __ldg(p.gfield + k), jx);
        jy = fmaf(rx, __ldg(p.gfield + p.fstride + k), jy);
        if (Q == 19) jz = fmaf(rx, __ldg(p.gfield + 2 * p.fstride + k), jz);
    }
    const float rn = 1.f + dd;
    const float uxn = jx / rn, uyn = jy / rn;
    stf(out + k, dd);
    stf(out + p.fstride + k, uxn);
    stf(out + 2 * p.fstride + k, uyn);
    if (Q == 19) stf(out + 3 * p.fstride + k, jz / rn);
    if (SC) stf(out + (Q == 19 ? 4 : 3) * p.fstride + k, fmaf(p.at, ldf(Tin + k), ts));
    if (BULK) stf(out + 3 * p.fstride + k, trs / rna - fmaf(uxn, uxn, uyn * uyn));
}

}  // namespace lwacm
