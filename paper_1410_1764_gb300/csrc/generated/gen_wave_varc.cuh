// GENERATED by paper_1410_1764_gb300.gen from the symbolic equation lists in
// gen/systems.py; do not edit.  Regenerate: python -m paper_1410_1764_gb300.gen
#pragma once

// variable-speed wave: u_t = rho, rho_t = s Lap u + grad s . grad u
// generated: 52 fp64 instructions, 64 algorithmic flops, 0 exp, 0 rcp per point
template <class LD, class SC>
__device__ __forceinline__ void chemora_varc_point(const LD& ld, const SC& sc, double (&out)[2]) {
  const double v_f1_0_0_0 = ld(1, 0, 0, 0);
  const double v_f2_2_0_0 = ld(2, 2, 0, 0);
  const double v_f2_m2_0_0 = ld(2, -2, 0, 0);
  const double t68 = v_f2_2_0_0 - v_f2_m2_0_0;
  const double v_f2_1_0_0 = ld(2, 1, 0, 0);
  const double v_f2_m1_0_0 = ld(2, -1, 0, 0);
  const double t65 = v_f2_1_0_0 - v_f2_m1_0_0;
  const double t73 = fma(8.0, t65, (-t68));
  const double t75 = sc.i12h * t73;
  const double v_f0_2_0_0 = ld(0, 2, 0, 0);
  const double v_f0_m2_0_0 = ld(0, -2, 0, 0);
  const double t77 = v_f0_2_0_0 - v_f0_m2_0_0;
  const double v_f0_1_0_0 = ld(0, 1, 0, 0);
  const double v_f0_m1_0_0 = ld(0, -1, 0, 0);
  const double t76 = v_f0_1_0_0 - v_f0_m1_0_0;
  const double t81 = fma(8.0, t76, (-t77));
  const double t83 = sc.i12h * t81;
  const double v_f2_0_2_0 = ld(2, 0, 2, 0);
  const double v_f2_0_m2_0 = ld(2, 0, -2, 0);
  const double t90 = v_f2_0_2_0 - v_f2_0_m2_0;
  const double v_f2_0_1_0 = ld(2, 0, 1, 0);
  const double v_f2_0_m1_0 = ld(2, 0, -1, 0);
  const double t87 = v_f2_0_1_0 - v_f2_0_m1_0;
  const double t94 = fma(8.0, t87, (-t90));
  const double t96 = sc.i12h * t94;
  const double v_f0_0_2_0 = ld(0, 0, 2, 0);
  const double v_f0_0_m2_0 = ld(0, 0, -2, 0);
  const double t98 = v_f0_0_2_0 - v_f0_0_m2_0;
  const double v_f0_0_1_0 = ld(0, 0, 1, 0);
  const double v_f0_0_m1_0 = ld(0, 0, -1, 0);
  const double t97 = v_f0_0_1_0 - v_f0_0_m1_0;
  const double t102 = fma(8.0, t97, (-t98));
  const double t104 = sc.i12h * t102;
  const double v_f2_0_0_2 = ld(2, 0, 0, 2);
  const double v_f2_0_0_m2 = ld(2, 0, 0, -2);
  const double t112 = v_f2_0_0_2 - v_f2_0_0_m2;
  const double v_f2_0_0_1 = ld(2, 0, 0, 1);
  const double v_f2_0_0_m1 = ld(2, 0, 0, -1);
  const double t109 = v_f2_0_0_1 - v_f2_0_0_m1;
  const double t116 = fma(8.0, t109, (-t112));
  const double t118 = sc.i12h * t116;
  const double v_f0_0_0_2 = ld(0, 0, 0, 2);
  const double v_f0_0_0_m2 = ld(0, 0, 0, -2);
  const double t120 = v_f0_0_0_2 - v_f0_0_0_m2;
  const double v_f0_0_0_1 = ld(0, 0, 0, 1);
  const double v_f0_0_0_m1 = ld(0, 0, 0, -1);
  const double t119 = v_f0_0_0_1 - v_f0_0_0_m1;
  const double t124 = fma(8.0, t119, (-t120));
  const double t126 = sc.i12h * t124;
  const double v_f0_0_0_0 = ld(0, 0, 0, 0);
  const double t16 = v_f0_2_0_0 - v_f0_0_0_0;
  const double t18 = v_f0_m2_0_0 - v_f0_0_0_0;
  const double t20 = t16 + t18;
  const double t8 = v_f0_1_0_0 - v_f0_0_0_0;
  const double t10 = v_f0_m1_0_0 - v_f0_0_0_0;
  const double t12 = t8 + t10;
  const double t24 = fma(16.0, t12, (-t20));
  const double t33 = v_f0_0_2_0 - v_f0_0_0_0;
  const double t35 = v_f0_0_m2_0 - v_f0_0_0_0;
  const double t37 = t33 + t35;
  const double t26 = v_f0_0_1_0 - v_f0_0_0_0;
  const double t28 = v_f0_0_m1_0 - v_f0_0_0_0;
  const double t30 = t26 + t28;
  const double t40 = fma(16.0, t30, (-t37));
  const double t50 = v_f0_0_0_2 - v_f0_0_0_0;
  const double t52 = v_f0_0_0_m2 - v_f0_0_0_0;
  const double t54 = t50 + t52;
  const double t43 = v_f0_0_0_1 - v_f0_0_0_0;
  const double t45 = v_f0_0_0_m1 - v_f0_0_0_0;
  const double t47 = t43 + t45;
  const double t57 = fma(16.0, t47, (-t54));
  const double t59 = t24 + t40 + t57;
  const double t62 = sc.i12h2 * t59;
  const double v_f2_0_0_0 = ld(2, 0, 0, 0);
  const double t132 = fma(t62, v_f2_0_0_0, fma(t118, t126, fma(t96, t104, t75 * t83)));
  out[0] = v_f1_0_0_0;
  out[1] = t132;
}
