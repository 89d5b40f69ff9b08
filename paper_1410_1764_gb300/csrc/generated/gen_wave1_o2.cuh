// GENERATED by paper_1410_1764_gb300.gen from the symbolic equation lists in
// gen/systems.py; do not edit.  Regenerate: python -m paper_1410_1764_gb300.gen
#pragma once

// scalar wave, first-order form of Eq. 1 (u, rho, v_i), order-2 D, from gen/wave1.eqs
// generated: 18 fp64 instructions, 20 algorithmic flops, 0 exp, 0 rcp per point
// out(v, value) receives output v (5 outputs) as soon as it is computed
template <class LD, class SC, class OUT>
__device__ __forceinline__ void chemora_wave1_o2_point(const LD& ld, const SC& sc, OUT& out) {
  const double v_f1_0_0_0 = ld(1, 0, 0, 0);
  const double v_f2_1_0_0 = ld(2, 1, 0, 0);
  const double v_f2_m1_0_0 = ld(2, -1, 0, 0);
  const double t67 = fma(v_f2_m1_0_0, -sc.k[0], v_f2_1_0_0);
  const double t13651 = fma(sc.k[7], t67, sc.k[1]);
  const double v_f3_0_1_0 = ld(3, 0, 1, 0);
  const double v_f3_0_m1_0 = ld(3, 0, -1, 0);
  const double t279 = fma(v_f3_0_m1_0, -sc.k[0], v_f3_0_1_0);
  const double t13654 = fma(sc.k[7], t279, sc.k[1]);
  const double v_f4_0_0_1 = ld(4, 0, 0, 1);
  const double v_f4_0_0_m1 = ld(4, 0, 0, -1);
  const double t327 = fma(v_f4_0_0_m1, -sc.k[0], v_f4_0_0_1);
  const double t13658 = fma(sc.k[7], t327, sc.k[1]);
  const double t13661 = fma(sc.ih, t13658, fma(sc.ih, t13654, fma(sc.ih, t13651, sc.k[1])));
  const double v_f1_1_0_0 = ld(1, 1, 0, 0);
  const double v_f1_m1_0_0 = ld(1, -1, 0, 0);
  const double t231 = fma(v_f1_m1_0_0, -sc.k[0], v_f1_1_0_0);
  const double t13663 = fma(sc.k[7], t231, sc.k[1]);
  const double t13665 = fma(sc.ih, t13663, sc.k[1]);
  const double v_f1_0_1_0 = ld(1, 0, 1, 0);
  const double v_f1_0_m1_0 = ld(1, 0, -1, 0);
  const double t243 = fma(v_f1_0_m1_0, -sc.k[0], v_f1_0_1_0);
  const double t13667 = fma(sc.k[7], t243, sc.k[1]);
  const double t13669 = fma(sc.ih, t13667, sc.k[1]);
  const double v_f1_0_0_1 = ld(1, 0, 0, 1);
  const double v_f1_0_0_m1 = ld(1, 0, 0, -1);
  const double t255 = fma(v_f1_0_0_m1, -sc.k[0], v_f1_0_0_1);
  const double t13671 = fma(sc.k[7], t255, sc.k[1]);
  const double t13673 = fma(sc.ih, t13671, sc.k[1]);
  out(0, v_f1_0_0_0);
  out(1, t13661);
  out(2, t13665);
  out(3, t13669);
  out(4, t13673);
}
