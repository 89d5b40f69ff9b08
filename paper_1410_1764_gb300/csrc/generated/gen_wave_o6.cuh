// GENERATED by paper_1410_1764_gb300.gen from the symbolic equation lists in
// gen/systems.py; do not edit.  Regenerate: python -m paper_1410_1764_gb300.gen
#pragma once

// scalar wave, two-variable form, order-6 Laplacian
// generated: 37 fp64 instructions, 45 algorithmic flops, 0 exp, 0 rcp per point
// out(v, value) receives output v (2 outputs) as soon as it is computed
template <class LD, class SC, class OUT>
__device__ __forceinline__ void chemora_wave_o6_point(const LD& ld, const SC& sc, OUT& out) {
  const double v_f1_0_0_0 = ld(1, 0, 0, 0);
  const double v_f0_1_0_0 = ld(0, 1, 0, 0);
  const double v_f0_0_0_0 = ld(0, 0, 0, 0);
  const double t10 = v_f0_1_0_0 - v_f0_0_0_0;
  const double v_f0_m1_0_0 = ld(0, -1, 0, 0);
  const double t12 = v_f0_m1_0_0 - v_f0_0_0_0;
  const double t14 = t10 + t12;
  const double v_f0_2_0_0 = ld(0, 2, 0, 0);
  const double t18 = v_f0_2_0_0 - v_f0_0_0_0;
  const double v_f0_m2_0_0 = ld(0, -2, 0, 0);
  const double t20 = v_f0_m2_0_0 - v_f0_0_0_0;
  const double t22 = t18 + t20;
  const double v_f0_0_1_0 = ld(0, 0, 1, 0);
  const double t28 = v_f0_0_1_0 - v_f0_0_0_0;
  const double v_f0_0_m1_0 = ld(0, 0, -1, 0);
  const double t30 = v_f0_0_m1_0 - v_f0_0_0_0;
  const double t32 = t28 + t30;
  const double v_f0_0_2_0 = ld(0, 0, 2, 0);
  const double t35 = v_f0_0_2_0 - v_f0_0_0_0;
  const double v_f0_0_m2_0 = ld(0, 0, -2, 0);
  const double t37 = v_f0_0_m2_0 - v_f0_0_0_0;
  const double t39 = t35 + t37;
  const double v_f0_0_0_1 = ld(0, 0, 0, 1);
  const double t45 = v_f0_0_0_1 - v_f0_0_0_0;
  const double v_f0_0_0_m1 = ld(0, 0, 0, -1);
  const double t47 = v_f0_0_0_m1 - v_f0_0_0_0;
  const double t49 = t45 + t47;
  const double v_f0_0_0_2 = ld(0, 0, 0, 2);
  const double t52 = v_f0_0_0_2 - v_f0_0_0_0;
  const double v_f0_0_0_m2 = ld(0, 0, 0, -2);
  const double t54 = v_f0_0_0_m2 - v_f0_0_0_0;
  const double t56 = t52 + t54;
  const double v_f0_3_0_0 = ld(0, 3, 0, 0);
  const double t5508 = v_f0_3_0_0 - v_f0_0_0_0;
  const double v_f0_m3_0_0 = ld(0, -3, 0, 0);
  const double t5510 = v_f0_m3_0_0 - v_f0_0_0_0;
  const double t5512 = t5508 + t5510;
  const double v_f0_0_3_0 = ld(0, 0, 3, 0);
  const double t5520 = v_f0_0_3_0 - v_f0_0_0_0;
  const double v_f0_0_m3_0 = ld(0, 0, -3, 0);
  const double t5522 = v_f0_0_m3_0 - v_f0_0_0_0;
  const double t5524 = t5520 + t5522;
  const double v_f0_0_0_3 = ld(0, 0, 0, 3);
  const double t5533 = v_f0_0_0_3 - v_f0_0_0_0;
  const double v_f0_0_0_m3 = ld(0, 0, 0, -3);
  const double t5535 = v_f0_0_0_m3 - v_f0_0_0_0;
  const double t5537 = t5533 + t5535;
  const double t13734 = fma(0.011111111111111112, t5537, fma(0.011111111111111112, t5524, fma(0.011111111111111112, t5512, fma(-0.15, t56, fma(1.5, t49, fma(-0.15, t39, fma(1.5, t32, fma(-0.15, t22, 1.5 * t14))))))));
  const double t13736 = sc.ih2 * t13734;
  out(0, v_f1_0_0_0);
  out(1, t13736);
}
