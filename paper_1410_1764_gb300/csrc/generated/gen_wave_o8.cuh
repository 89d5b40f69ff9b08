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
  const double t10 = fma(v_f0_0_0_0, -sc.k[0], v_f0_1_0_0);
  const double v_f0_m1_0_0 = ld(0, -1, 0, 0);
  const double t12 = fma(v_f0_0_0_0, -sc.k[0], v_f0_m1_0_0);
  const double t14 = fma(t12, sc.k[0], t10);
  const double v_f0_2_0_0 = ld(0, 2, 0, 0);
  const double t18 = fma(v_f0_0_0_0, -sc.k[0], v_f0_2_0_0);
  const double v_f0_m2_0_0 = ld(0, -2, 0, 0);
  const double t20 = fma(v_f0_0_0_0, -sc.k[0], v_f0_m2_0_0);
  const double t22 = fma(t20, sc.k[0], t18);
  const double v_f0_0_1_0 = ld(0, 0, 1, 0);
  const double t28 = fma(v_f0_0_0_0, -sc.k[0], v_f0_0_1_0);
  const double v_f0_0_m1_0 = ld(0, 0, -1, 0);
  const double t30 = fma(v_f0_0_0_0, -sc.k[0], v_f0_0_m1_0);
  const double t32 = fma(t30, sc.k[0], t28);
  const double v_f0_0_2_0 = ld(0, 0, 2, 0);
  const double t35 = fma(v_f0_0_0_0, -sc.k[0], v_f0_0_2_0);
  const double v_f0_0_m2_0 = ld(0, 0, -2, 0);
  const double t37 = fma(v_f0_0_0_0, -sc.k[0], v_f0_0_m2_0);
  const double t39 = fma(t37, sc.k[0], t35);
  const double v_f0_0_0_1 = ld(0, 0, 0, 1);
  const double t45 = fma(v_f0_0_0_0, -sc.k[0], v_f0_0_0_1);
  const double v_f0_0_0_m1 = ld(0, 0, 0, -1);
  const double t47 = fma(v_f0_0_0_0, -sc.k[0], v_f0_0_0_m1);
  const double t49 = fma(t47, sc.k[0], t45);
  const double v_f0_0_0_2 = ld(0, 0, 0, 2);
  const double t52 = fma(v_f0_0_0_0, -sc.k[0], v_f0_0_0_2);
  const double v_f0_0_0_m2 = ld(0, 0, 0, -2);
  const double t54 = fma(v_f0_0_0_0, -sc.k[0], v_f0_0_0_m2);
  const double t56 = fma(t54, sc.k[0], t52);
  const double v_f0_3_0_0 = ld(0, 3, 0, 0);
  const double t5508 = fma(v_f0_0_0_0, -sc.k[0], v_f0_3_0_0);
  const double v_f0_m3_0_0 = ld(0, -3, 0, 0);
  const double t5510 = fma(v_f0_0_0_0, -sc.k[0], v_f0_m3_0_0);
  const double t5512 = fma(t5510, sc.k[0], t5508);
  const double v_f0_0_3_0 = ld(0, 0, 3, 0);
  const double t5520 = fma(v_f0_0_0_0, -sc.k[0], v_f0_0_3_0);
  const double v_f0_0_m3_0 = ld(0, 0, -3, 0);
  const double t5522 = fma(v_f0_0_0_0, -sc.k[0], v_f0_0_m3_0);
  const double t5524 = fma(t5522, sc.k[0], t5520);
  const double v_f0_0_0_3 = ld(0, 0, 0, 3);
  const double t5533 = fma(v_f0_0_0_0, -sc.k[0], v_f0_0_0_3);
  const double v_f0_0_0_m3 = ld(0, 0, 0, -3);
  const double t5535 = fma(v_f0_0_0_0, -sc.k[0], v_f0_0_0_m3);
  const double t5537 = fma(t5535, sc.k[0], t5533);
  const double v_f0_4_0_0 = ld(0, 4, 0, 0);
  const double t13793 = fma(v_f0_0_0_0, -sc.k[0], v_f0_4_0_0);
  const double v_f0_m4_0_0 = ld(0, -4, 0, 0);
  const double t13795 = fma(v_f0_0_0_0, -sc.k[0], v_f0_m4_0_0);
  const double t13797 = fma(t13795, sc.k[0], t13793);
  const double v_f0_0_4_0 = ld(0, 0, 4, 0);
  const double t13811 = fma(v_f0_0_0_0, -sc.k[0], v_f0_0_4_0);
  const double v_f0_0_m4_0 = ld(0, 0, -4, 0);
  const double t13813 = fma(v_f0_0_0_0, -sc.k[0], v_f0_0_m4_0);
  const double t13815 = fma(t13813, sc.k[0], t13811);
  const double v_f0_0_0_4 = ld(0, 0, 0, 4);
  const double t13826 = fma(v_f0_0_0_0, -sc.k[0], v_f0_0_0_4);
  const double v_f0_0_0_m4 = ld(0, 0, 0, -4);
  const double t13828 = fma(v_f0_0_0_0, -sc.k[0], v_f0_0_0_m4);
  const double t13830 = fma(t13828, sc.k[0], t13826);
  const double t13840 = fma(-sc.k[25], t13830, fma(-sc.k[25], t13815, fma(-sc.k[25], t13797, fma(sc.k[24], t5537, fma(sc.k[24], t5524, fma(sc.k[24], t5512, fma(-sc.k[23], t56, fma(sc.k[22], t49, fma(-sc.k[23], t39, fma(sc.k[22], t32, fma(-sc.k[23], t22, fma(sc.k[22], t14, sc.k[1]))))))))))));
  const double t13842 = fma(sc.ih2, t13840, sc.k[1]);
  out(0, v_f1_0_0_0);
  out(1, t13842);
}
