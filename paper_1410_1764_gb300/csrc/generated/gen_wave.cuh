// GENERATED by paper_1410_1764_gb300.gen from the symbolic equation lists in
// gen/systems.py; do not edit.  Regenerate: python -m paper_1410_1764_gb300.gen
#pragma once

// scalar wave, Eq. 1 two-variable form: u_t = rho, rho_t = Lap u
// generated: 24 fp64 instructions, 27 algorithmic flops, 0 exp, 0 rcp per point
// out(v, value) receives output v (2 outputs) as soon as it is computed
template <class LD, class SC, class OUT>
__device__ __forceinline__ void chemora_wave_point(const LD& ld, const SC& sc, OUT& out) {
  const double v_f1_0_0_0 = ld(1, 0, 0, 0);
  const double v_f0_2_0_0 = ld(0, 2, 0, 0);
  const double v_f0_0_0_0 = ld(0, 0, 0, 0);
  const double t18 = v_f0_2_0_0 - v_f0_0_0_0;
  const double v_f0_m2_0_0 = ld(0, -2, 0, 0);
  const double t20 = v_f0_m2_0_0 - v_f0_0_0_0;
  const double v_f0_0_2_0 = ld(0, 0, 2, 0);
  const double t35 = v_f0_0_2_0 - v_f0_0_0_0;
  const double v_f0_0_m2_0 = ld(0, 0, -2, 0);
  const double t37 = v_f0_0_m2_0 - v_f0_0_0_0;
  const double v_f0_0_0_2 = ld(0, 0, 0, 2);
  const double t52 = v_f0_0_0_2 - v_f0_0_0_0;
  const double v_f0_0_0_m2 = ld(0, 0, 0, -2);
  const double t54 = v_f0_0_0_m2 - v_f0_0_0_0;
  const double v_f0_1_0_0 = ld(0, 1, 0, 0);
  const double t10 = v_f0_1_0_0 - v_f0_0_0_0;
  const double v_f0_m1_0_0 = ld(0, -1, 0, 0);
  const double t12 = v_f0_m1_0_0 - v_f0_0_0_0;
  const double t14 = t10 + t12;
  const double v_f0_0_1_0 = ld(0, 0, 1, 0);
  const double t28 = v_f0_0_1_0 - v_f0_0_0_0;
  const double v_f0_0_m1_0 = ld(0, 0, -1, 0);
  const double t30 = v_f0_0_m1_0 - v_f0_0_0_0;
  const double t32 = t28 + t30;
  const double v_f0_0_0_1 = ld(0, 0, 0, 1);
  const double t45 = v_f0_0_0_1 - v_f0_0_0_0;
  const double v_f0_0_0_m1 = ld(0, 0, 0, -1);
  const double t47 = v_f0_0_0_m1 - v_f0_0_0_0;
  const double t49 = t45 + t47;
  const double t61 = fma(16.0, t49, fma(16.0, t32, fma(16.0, t14, (-t18) - t20 - t35 - t37 - t52 - t54)));
  const double t64 = sc.i12h2 * t61;
  out(0, v_f1_0_0_0);
  out(1, t64);
}
