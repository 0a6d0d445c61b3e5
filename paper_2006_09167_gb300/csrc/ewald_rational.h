/* Generated by gen_ewald_rational.py -- do not edit.
 * Rational approximations, z = beta r, on 0 <= z <= ZMAX of
 *   H(z) = (erf(z)/z - 2/sqrt(pi) exp(-z^2)) / z^2   (in s = z^2/ZMAX^2)
 *   X(z) = exp(z^2) erfc(z)                          (in t = z/ZMAX)
 * and exp(w) = 1 + w (C1 + C2 w + ...) on |w| <= ln2/2 with the Cody-Waite
 * constants of exp(-x) = 2^-n exp(-(x - n ln2)).
 * Relative errors below are measured against mpmath / FP64.
 */
#pragma once
#define NB_EW_ZMAX 4.0f
/* H: degrees (6,5); fp64: max rel err 6.29e-08; fp32 Horner max rel err 3.47e-07, mean -1.41e-08 */
#define NB_EW_HP0 0.7522528171539307f
#define NB_EW_HP1 -0.5743048191070557f
#define NB_EW_HP2 4.628017902374268f
#define NB_EW_HP3 -0.8285208940505981f
#define NB_EW_HP4 3.300889492034912f
#define NB_EW_HP5 -1.0783452987670898f
#define NB_EW_HP6 0.18139305710792542f
#define NB_EW_HQ1 8.836585998535156f
#define NB_EW_HQ2 36.12339401245117f
#define NB_EW_HQ3 88.59178924560547f
#define NB_EW_HQ4 137.36947631835938f
#define NB_EW_HQ5 136.4874267578125f
/* X: degrees (6,6); FP32 coefficients, exact evaluation: max rel err 2.88e-09; fp32 Horner max rel err 3.6e-07, mean 5.81e-09 */
#define NB_EW_XP0 1.0f
#define NB_EW_XP1 5.064917087554932f
#define NB_EW_XP2 12.871368408203125f
#define NB_EW_XP3 18.6243839263916f
#define NB_EW_XP4 15.265811920166016f
#define NB_EW_XP5 5.703533172607422f
#define NB_EW_XP6 0.0005424104747362435f
#define NB_EW_XQ1 9.578433990478516f
#define NB_EW_XQ2 40.103782653808594f
#define NB_EW_XQ3 94.52271270751953f
#define NB_EW_XQ4 133.38247680664062f
#define NB_EW_XQ5 108.19001007080078f
#define NB_EW_XQ6 40.45461654663086f
/* exp: degree 7; fp64 max rel err 4.67e-11; fp32 exp(-x) on [0,16] max rel err 7.23e-08, mean -1.8e-10 */
#define NB_EXP_LOG2E 1.4426950216293335f
#define NB_EXP_LN2_HI 0.693145751953125f
#define NB_EXP_LN2_LO 1.428606765330187e-06f
#define NB_EXP_C1 1.0f
#define NB_EXP_C2 0.5f
#define NB_EXP_C3 0.1666666567325592f
#define NB_EXP_C4 0.04166627302765846f
#define NB_EXP_C5 0.008333568461239338f
#define NB_EXP_C6 0.0013945897808298469f
#define NB_EXP_C7 0.0001976766943698749f
