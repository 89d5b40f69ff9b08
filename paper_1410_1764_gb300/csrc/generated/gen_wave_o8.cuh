// GENERATED by paper_1410_1764_gb300.gen from the symbolic equation lists in
// gen/systems.py; do not edit.  Regenerate: python -m paper_1410_1764_gb300.gen
#pragma once

// scalar wave, two-variable form, order-8 Laplacian
// generated: 49 fp64 instructions, 60 algorithmic flops, 0 exp, 0 rcp per point
// out(v, value) receives output v (2 outputs) as soon as it is computed
template <class LD, class SC, class OUT>
__device__ __forceinline__ void chemora_wave_o8_point(const LD& ld, const SC& sc, OUT& out) {
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
  const double v_f0_4_0_0 = ld(0, 4, 0, 0);
  const double t13793 = v_f0_4_0_0 - v_f0_0_0_0;
  const double v_f0_m4_0_0 = ld(0, -4, 0, 0);
  const double t13795 = v_f0_m4_0_0 - v_f0_0_0_0;
  const double t13797 = t13793 + t13795;
  const double v_f0_0_4_0 = ld(0, 0, 4, 0);
  const double t13811 = v_f0_0_4_0 - v_f0_0_0_0;
  const double v_f0_0_m4_0 = ld(0, 0, -4, 0);
  const double t13813 = v_f0_0_m4_0 - v_f0_0_0_0;
  const double t13815 = t13811 + t13813;
  const double v_f0_0_0_4 = ld(0, 0, 0, 4);
  const double t13826 = v_f0_0_0_4 - v_f0_0_0_0;
  const double v_f0_0_0_m4 = ld(0, 0, 0, -4);
  const double t13828 = v_f0_0_0_m4 - v_f0_0_0_0;
  const double t13830 = t13826 + t13828;
  const double t13840 = fma(-0.0017857142857142857, t13830, fma(-0.0017857142857142857, t13815, fma(-0.0017857142857142857, t13797, fma(0.025396825396825397, t5537, fma(0.025396825396825397, t5524, fma(0.025396825396825397, t5512, fma(-0.2, t56, fma(1.6, t49, fma(-0.2, t39, fma(1.6, t32, fma(-0.2, t22, 1.6 * t14)))))))))));
  const double t13842 = sc.ih2 * t13840;
  out(0, v_f1_0_0_0);
  out(1, t13842);
}
