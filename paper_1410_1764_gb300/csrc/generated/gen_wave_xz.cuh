// GENERATED by paper_1410_1764_gb300.gen from the symbolic equation lists in
// gen/systems.py; do not edit.  Regenerate: python -m paper_1410_1764_gb300.gen
#pragma once

// scalar wave as chemora_wave_point, x-direction differences shared across warp lanes and the z-direction second difference from a register queue of z first differences kept by a thread marching along z
// generated: 16 fp64 instructions, 19 algorithmic flops, 0 exp, 0 rcp per point
// out(v, value) receives output v (2 outputs) as soon as it is computed
template <class LD, class SC, class OUT>
__device__ __forceinline__ void chemora_wave_xz_point(const LD& ld, const SC& sc, OUT& out) {
  const double v_f1_0_0_0 = ld(1, 0, 0, 0);
  const double v_f0_0_2_0 = ld(0, 0, 2, 0);
  const double v_f0_0_0_0 = ld(0, 0, 0, 0);
  const double t35 = fma(v_f0_0_0_0, -sc.k[0], v_f0_0_2_0);
  const double v_f0_0_m2_0 = ld(0, 0, -2, 0);
  const double t37 = fma(v_f0_0_0_0, -sc.k[0], v_f0_0_m2_0);
  const double v_f0_1_0_0 = ld(0, 1, 0, 0);
  const double t10 = fma(v_f0_0_0_0, -sc.k[0], v_f0_1_0_0);
  const double t6654 = ld.ext_dx(0, sc.k[0]);
  const double t6658 = chemora_xshfl(t10, t6654, 1, 3);
  const double t6659 = chemora_xshfl(t10, t6654, -2, 3);
  const double t6992 = fma(t6659, -sc.k[0], t6658);
  const double v_zqb_0 = ld.qb[0];
  const double v_f0_0_1_0 = ld(0, 0, 1, 0);
  const double t28 = fma(v_f0_0_0_0, -sc.k[0], v_f0_0_1_0);
  const double v_f0_0_m1_0 = ld(0, 0, -1, 0);
  const double t30 = fma(v_f0_0_0_0, -sc.k[0], v_f0_0_m1_0);
  const double t32 = fma(t30, sc.k[0], t28);
  const double t6655 = chemora_xshfl(t10, t6654, -1, 3);
  const double t6991 = fma(t6655, -sc.k[0], t10);
  const double v_zqa_0 = ld.qa[0];
  const double t13932 = fma(sc.k[12], v_zqa_0, fma(sc.k[12], t6991, fma(sc.k[4], t32, fma(v_zqb_0, -sc.k[0], fma(t6992, -sc.k[0], fma(t37, -sc.k[0], (-t35)))))));
  const double t13934 = fma(sc.i12h2, t13932, sc.k[1]);
  out(0, v_f1_0_0_0);
  out(1, t13934);
}
