// GENERATED by paper_1410_1764_gb300.gen from the symbolic equation lists in
// gen/systems.py; do not edit.  Regenerate: python -m paper_1410_1764_gb300.gen
#pragma once

// variable-speed wave: u_t = rho, rho_t = s Lap u + G . grad u, with s = c^2 and G = grad s read from grid functions 2 and 3-5
// generated: 40 fp64 instructions, 49 algorithmic flops, 0 exp, 0 rcp per point
// out(v, value) receives output v (2 outputs) as soon as it is computed
template <class LD, class SC, class OUT>
__device__ __forceinline__ void chemora_varc_point(const LD& ld, const SC& sc, OUT& out) {
  const double v_f1_0_0_0 = ld(1, 0, 0, 0);
  const double v_f0_2_0_0 = ld(0, 2, 0, 0);
  const double v_f0_0_0_0 = ld(0, 0, 0, 0);
  const double t18 = fma(v_f0_0_0_0, -sc.k[0], v_f0_2_0_0);
  const double v_f0_m2_0_0 = ld(0, -2, 0, 0);
  const double t20 = fma(v_f0_0_0_0, -sc.k[0], v_f0_m2_0_0);
  const double v_f0_0_2_0 = ld(0, 0, 2, 0);
  const double t35 = fma(v_f0_0_0_0, -sc.k[0], v_f0_0_2_0);
  const double v_f0_0_m2_0 = ld(0, 0, -2, 0);
  const double t37 = fma(v_f0_0_0_0, -sc.k[0], v_f0_0_m2_0);
  const double v_f0_0_0_2 = ld(0, 0, 0, 2);
  const double t52 = fma(v_f0_0_0_0, -sc.k[0], v_f0_0_0_2);
  const double v_f0_0_0_m2 = ld(0, 0, 0, -2);
  const double t54 = fma(v_f0_0_0_0, -sc.k[0], v_f0_0_0_m2);
  const double v_f0_1_0_0 = ld(0, 1, 0, 0);
  const double t10 = fma(v_f0_0_0_0, -sc.k[0], v_f0_1_0_0);
  const double v_f0_m1_0_0 = ld(0, -1, 0, 0);
  const double t12 = fma(v_f0_0_0_0, -sc.k[0], v_f0_m1_0_0);
  const double t14 = fma(t12, sc.k[0], t10);
  const double v_f0_0_1_0 = ld(0, 0, 1, 0);
  const double t28 = fma(v_f0_0_0_0, -sc.k[0], v_f0_0_1_0);
  const double v_f0_0_m1_0 = ld(0, 0, -1, 0);
  const double t30 = fma(v_f0_0_0_0, -sc.k[0], v_f0_0_m1_0);
  const double t32 = fma(t30, sc.k[0], t28);
  const double v_f0_0_0_1 = ld(0, 0, 0, 1);
  const double t45 = fma(v_f0_0_0_0, -sc.k[0], v_f0_0_0_1);
  const double v_f0_0_0_m1 = ld(0, 0, 0, -1);
  const double t47 = fma(v_f0_0_0_0, -sc.k[0], v_f0_0_0_m1);
  const double t49 = fma(t47, sc.k[0], t45);
  const double t61 = fma(sc.k[4], t49, fma(sc.k[4], t32, fma(sc.k[4], t14, fma(t54, -sc.k[0], fma(t52, -sc.k[0], fma(t37, -sc.k[0], fma(t35, -sc.k[0], fma(t20, -sc.k[0], (-t18)))))))));
  const double t64 = fma(sc.i12h2, t61, sc.k[1]);
  const double v_f2_0_0_0 = ld(2, 0, 0, 0);
  const double t79 = fma(v_f0_m2_0_0, -sc.k[0], v_f0_2_0_0);
  const double t78 = fma(v_f0_m1_0_0, -sc.k[0], v_f0_1_0_0);
  const double t83 = fma(sc.k[3], t78, (-t79));
  const double t85 = fma(sc.i12h, t83, sc.k[1]);
  const double v_f3_0_0_0 = ld(3, 0, 0, 0);
  const double t100 = fma(v_f0_0_m2_0, -sc.k[0], v_f0_0_2_0);
  const double t99 = fma(v_f0_0_m1_0, -sc.k[0], v_f0_0_1_0);
  const double t104 = fma(sc.k[3], t99, (-t100));
  const double t106 = fma(sc.i12h, t104, sc.k[1]);
  const double v_f4_0_0_0 = ld(4, 0, 0, 0);
  const double t122 = fma(v_f0_0_0_m2, -sc.k[0], v_f0_0_0_2);
  const double t121 = fma(v_f0_0_0_m1, -sc.k[0], v_f0_0_0_1);
  const double t126 = fma(sc.k[3], t121, (-t122));
  const double t128 = fma(sc.i12h, t126, sc.k[1]);
  const double v_f5_0_0_0 = ld(5, 0, 0, 0);
  const double t13941 = fma(t128, v_f5_0_0_0, fma(t106, v_f4_0_0_0, fma(t85, v_f3_0_0_0, fma(t64, v_f2_0_0_0, sc.k[1]))));
  out(0, v_f1_0_0_0);
  out(1, t13941);
}
