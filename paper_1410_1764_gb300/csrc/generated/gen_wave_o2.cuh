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
  const double t10 = fma(v_f0_0_0_0, -sc.k[0], v_f0_1_0_0);
  const double v_f0_m1_0_0 = ld(0, -1, 0, 0);
  const double t12 = fma(v_f0_0_0_0, -sc.k[0], v_f0_m1_0_0);
  const double v_f0_0_1_0 = ld(0, 0, 1, 0);
  const double t28 = fma(v_f0_0_0_0, -sc.k[0], v_f0_0_1_0);
  const double v_f0_0_m1_0 = ld(0, 0, -1, 0);
  const double t30 = fma(v_f0_0_0_0, -sc.k[0], v_f0_0_m1_0);
  const double v_f0_0_0_1 = ld(0, 0, 0, 1);
  const double t45 = fma(v_f0_0_0_0, -sc.k[0], v_f0_0_0_1);
  const double v_f0_0_0_m1 = ld(0, 0, 0, -1);
  const double t47 = fma(v_f0_0_0_0, -sc.k[0], v_f0_0_0_m1);
  const double t13647 = fma(t47, sc.k[0], fma(t45, sc.k[0], fma(t30, sc.k[0], fma(t28, sc.k[0], fma(t12, sc.k[0], t10)))));
  const double t13649 = fma(sc.ih2, t13647, sc.k[1]);
  out(0, v_f1_0_0_0);
  out(1, t13649);
}
