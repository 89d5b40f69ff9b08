// GENERATED by paper_1410_1764_gb300.gen from the symbolic equation lists in
// gen/systems.py; do not edit.  Regenerate: python -m paper_1410_1764_gb300.gen
#pragma once
// Numeric constants of the generated point bodies, read at run time from
// Scalars::k (a kernel parameter) so that every FP64 operation is an fma
// with register or constant-bank operands.
#define CHEMORA_NK 29
#define CHEMORA_K_ONE 0
#define CHEMORA_K_MZERO 1
#define CHEMORA_K_TWO 2
#define CHEMORA_K_EIGHT 3
#if !defined(__CUDACC_RTC__)
static const double kChemoraK[CHEMORA_NK] = {
    0x1.0000000000000p+0,  // 0: 1.0
    -0.0,  // 1: -0.0
    0x1.0000000000000p+1,  // 2: 2.0
    0x1.0000000000000p+3,  // 3: 8.0
    0x1.0000000000000p+4,  // 4: 16.0
    0x1.5555555555555p-1,  // 5: 0.6666666666666666
    0x1.0000000000000p+2,  // 6: 4.0
    0x1.0000000000000p-1,  // 7: 0.5
    0x1.5555555555555p-3,  // 8: 0.16666666666666666
    0x1.8000000000000p+1,  // 9: 3.0
    0x1.5555555555555p-2,  // 10: 0.3333333333333333
    0x1.8000000000000p+2,  // 11: 6.0
    0x1.e000000000000p+3,  // 12: 15.0
    0x1.5555555555555p-4,  // 13: 0.08333333333333333
    0x1.8000000000000p-1,  // 14: 0.75
    0x1.c000000000000p+2,  // 15: 7.0
    0x1.4000000000000p+3,  // 16: 10.0
    0x1.4000000000000p+2,  // 17: 5.0
    0x1.8000000000000p+0,  // 18: 1.5
    0x1.3333333333333p-3,  // 19: 0.15
    0x1.6c16c16c16c17p-7,  // 20: 0.011111111111111112
    0x1.1111111111111p-6,  // 21: 0.016666666666666666
    0x1.999999999999ap+0,  // 22: 1.6
    0x1.999999999999ap-3,  // 23: 0.2
    0x1.a01a01a01a01ap-6,  // 24: 0.025396825396825397
    0x1.d41d41d41d41dp-10,  // 25: 0.0017857142857142857
    0x1.999999999999ap-1,  // 26: 0.8
    0x1.3813813813814p-5,  // 27: 0.0380952380952381
    0x1.d41d41d41d41dp-9,  // 28: 0.0035714285714285713
};
#endif
