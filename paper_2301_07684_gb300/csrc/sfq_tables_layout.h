#pragma once
// Generated by paper_2301_07684_gb300/fitgen/generate.py -- do not edit.
// Piecewise monomial (Horner) coefficients in the local variable of each piece;
// see the generator for the layout and the fitted functions.

// nlc_rate_f64: max relative fit error 1.828e-12 (target 5.0e-12)
#define NLC_RATE_F64_X_ELO -10
#define NLC_RATE_F64_X_EHI 20
#define NLC_RATE_F64_X_SUB 1
#define NLC_RATE_F64_X_LOW 1
#define NLC_RATE_F64_X_SUBLOW 0
#define NLC_RATE_F64_X_NPIECES 61
#define NLC_RATE_F64_DEG 10
#define NLC_RATE_F64_COUNT 671
#define NLC_RATE_F64_ERR 1.828e-12

// nlc_rate_f32: max relative fit error 2.558e-08 (target 5.0e-08)
#define NLC_RATE_F32_X_ELO -10
#define NLC_RATE_F32_X_EHI 20
#define NLC_RATE_F32_X_SUB 0
#define NLC_RATE_F32_X_LOW 1
#define NLC_RATE_F32_X_SUBLOW 0
#define NLC_RATE_F32_X_NPIECES 31
#define NLC_RATE_F32_DEG 8
#define NLC_RATE_F32_COUNT 279
#define NLC_RATE_F32_ERR 2.558e-08

// nbw_rate_f64: max relative fit error 1.796e-12 (target 5.0e-12)
#define NBW_RATE_F64_X_ELO -7
#define NBW_RATE_F64_X_EHI 20
#define NBW_RATE_F64_X_SUB 1
#define NBW_RATE_F64_X_LOW 0
#define NBW_RATE_F64_X_SUBLOW 0
#define NBW_RATE_F64_X_NPIECES 54
#define NBW_RATE_F64_DEG 10
#define NBW_RATE_F64_COUNT 594
#define NBW_RATE_F64_ERR 1.796e-12

// nbw_rate_f32: max relative fit error 2.645e-08 (target 5.0e-08)
#define NBW_RATE_F32_X_ELO -7
#define NBW_RATE_F32_X_EHI 20
#define NBW_RATE_F32_X_SUB 0
#define NBW_RATE_F32_X_LOW 0
#define NBW_RATE_F32_X_SUBLOW 0
#define NBW_RATE_F32_X_NPIECES 27
#define NBW_RATE_F32_DEG 8
#define NBW_RATE_F32_COUNT 243
#define NBW_RATE_F32_ERR 2.645e-08

// k23_f64: max relative fit error 2.710e-12 (target 5.0e-12)
#define K23_F64_X_ELO -64
#define K23_F64_X_EHI 12
#define K23_F64_X_SUB 1
#define K23_F64_X_LOW 0
#define K23_F64_X_SUBLOW 0
#define K23_F64_X_NPIECES 152
#define K23_F64_DEG 9
#define K23_F64_COUNT 1520
#define K23_F64_ERR 2.710e-12

// k23_f32: max relative fit error 3.847e-09 (target 5.0e-08)
#define K23_F32_X_ELO -64
#define K23_F32_X_EHI 12
#define K23_F32_X_SUB 0
#define K23_F32_X_LOW 0
#define K23_F32_X_SUBLOW 0
#define K23_F32_X_NPIECES 76
#define K23_F32_DEG 8
#define K23_F32_COUNT 684
#define K23_F32_ERR 3.847e-09

// ki13_f64: max relative fit error 4.008e-12 (target 5.0e-12)
#define KI13_F64_X_ELO -64
#define KI13_F64_X_EHI 12
#define KI13_F64_X_SUB 1
#define KI13_F64_X_LOW 0
#define KI13_F64_X_SUBLOW 0
#define KI13_F64_X_NPIECES 152
#define KI13_F64_DEG 10
#define KI13_F64_COUNT 1672
#define KI13_F64_ERR 4.008e-12

// ki13_f32: max relative fit error 8.705e-09 (target 5.0e-08)
#define KI13_F32_X_ELO -64
#define KI13_F32_X_EHI 12
#define KI13_F32_X_SUB 0
#define KI13_F32_X_LOW 0
#define KI13_F32_X_SUBLOW 0
#define KI13_F32_X_NPIECES 76
#define KI13_F32_DEG 9
#define KI13_F32_COUNT 760
#define KI13_F32_ERR 8.705e-09

// nlc_inv_f64: max relative fit error 4.734e-13 (target 5.0e-12)
#define NLC_INV_F64_X_ELO -10
#define NLC_INV_F64_X_EHI 12
#define NLC_INV_F64_X_SUB 1
#define NLC_INV_F64_X_LOW 1
#define NLC_INV_F64_X_SUBLOW 0
#define NLC_INV_F64_X_NPIECES 45
#define NLC_INV_F64_Y_ELO -6
#define NLC_INV_F64_Y_EHI 0
#define NLC_INV_F64_Y_SUB 1
#define NLC_INV_F64_Y_LOW 1
#define NLC_INV_F64_Y_SUBLOW 0
#define NLC_INV_F64_Y_NPIECES 57
#define NLC_INV_F64_Y_QLO -24
#define NLC_INV_F64_Y_SUBQ 1
#define NLC_INV_F64_DX 11
#define NLC_INV_F64_DY 11
#define NLC_INV_F64_COUNT 369360
#define NLC_INV_F64_ERR 4.734e-13

// nlc_inv_f32: max relative fit error 6.945e-08 (target 3.0e-07)
#define NLC_INV_F32_X_ELO -10
#define NLC_INV_F32_X_EHI 12
#define NLC_INV_F32_X_SUB 0
#define NLC_INV_F32_X_LOW 1
#define NLC_INV_F32_X_SUBLOW 0
#define NLC_INV_F32_X_NPIECES 23
#define NLC_INV_F32_Y_ELO -6
#define NLC_INV_F32_Y_EHI 0
#define NLC_INV_F32_Y_SUB 0
#define NLC_INV_F32_Y_LOW 1
#define NLC_INV_F32_Y_SUBLOW 0
#define NLC_INV_F32_Y_NPIECES 29
#define NLC_INV_F32_Y_QLO -24
#define NLC_INV_F32_Y_SUBQ 0
#define NLC_INV_F32_DX 8
#define NLC_INV_F32_DY 8
#define NLC_INV_F32_COUNT 54027
#define NLC_INV_F32_ERR 6.945e-08

// nbw_inv_f64: max relative fit error 1.808e-12 (target 5.0e-12)
#define NBW_INV_F64_X_ELO -7
#define NBW_INV_F64_X_EHI 12
#define NBW_INV_F64_X_SUB 1
#define NBW_INV_F64_X_LOW 0
#define NBW_INV_F64_X_SUBLOW 0
#define NBW_INV_F64_X_NPIECES 38
#define NBW_INV_F64_Y_ELO -6
#define NBW_INV_F64_Y_EHI 0
#define NBW_INV_F64_Y_SUB 1
#define NBW_INV_F64_Y_LOW 1
#define NBW_INV_F64_Y_SUBLOW 0
#define NBW_INV_F64_Y_NPIECES 55
#define NBW_INV_F64_Y_QLO -23
#define NBW_INV_F64_Y_SUBQ 1
#define NBW_INV_F64_DX 11
#define NBW_INV_F64_DY 11
#define NBW_INV_F64_COUNT 300960
#define NBW_INV_F64_ERR 1.808e-12

// nbw_inv_f32: max relative fit error 2.162e-07 (target 3.0e-07)
#define NBW_INV_F32_X_ELO -7
#define NBW_INV_F32_X_EHI 12
#define NBW_INV_F32_X_SUB 0
#define NBW_INV_F32_X_LOW 0
#define NBW_INV_F32_X_SUBLOW 0
#define NBW_INV_F32_X_NPIECES 19
#define NBW_INV_F32_Y_ELO -6
#define NBW_INV_F32_Y_EHI 0
#define NBW_INV_F32_Y_SUB 0
#define NBW_INV_F32_Y_LOW 1
#define NBW_INV_F32_Y_SUBLOW 0
#define NBW_INV_F32_Y_NPIECES 28
#define NBW_INV_F32_Y_QLO -23
#define NBW_INV_F32_Y_SUBQ 0
#define NBW_INV_F32_DX 8
#define NBW_INV_F32_DY 8
#define NBW_INV_F32_COUNT 43092
#define NBW_INV_F32_ERR 2.162e-07

