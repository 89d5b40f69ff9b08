// GENERATED by paper_1410_1764_gb300.gen from the symbolic equation lists in
// gen/systems.py; do not edit.  Regenerate: python -m paper_1410_1764_gb300.gen
#pragma once

// scalar wave, two-variable form, order-2 Laplacian
// generated: 12 fp64 instructions, 12 algorithmic flops, 0 exp, 0 rcp per point
// out(v, value) receives output v (2 outputs) as soon as it is computed
template <class LD, class SC, class OUT>
__device__ __forceinline__ void chemora_wave_o2_point(const LD& ld, const SC& sc, OUT& out) {
  const double v_f1_0_0_0 = ld(1, 0, 0, 0);
  const double v_f0_1_0_0 = ld(0, 1, 0, 0);
  const double v_f0_0_0_0 = ld(0, 0, 0, 0);
  const double t10 = v_f0_1_0_0 - v_f0_0_0_0;
  const double v_f0_m1_0_0 = ld(0, -1, 0, 0);
  const double t12 = v_f0_m1_0_0 - v_f0_0_0_0;
  const double v_f0_0_1_0 = ld(0, 0, 1, 0);
  const double t28 = v_f0_0_1_0 - v_f0_0_0_0;
  const double v_f0_0_m1_0 = ld(0, 0, -1, 0);
  const double t30 = v_f0_0_m1_0 - v_f0_0_0_0;
  const double v_f0_0_0_1 = ld(0, 0, 0, 1);
  const double t45 = v_f0_0_0_1 - v_f0_0_0_0;
  const double v_f0_0_0_m1 = ld(0, 0, 0, -1);
  const double t47 = v_f0_0_0_m1 - v_f0_0_0_0;
  const double t13647 = t10 + t12 + t28 + t30 + t45 + t47;
  const double t13649 = sc.ih2 * t13647;
  out(0, v_f1_0_0_0);
  out(1, t13649);
}
