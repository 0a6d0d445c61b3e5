/* Generated by gen_ewald_rational.py -- do not edit.
 * Rational approximations, z = beta r, of
 *   H(z) = (erf(z)/z - 2/sqrt(pi) exp(-z^2)) / z^2 and E(z) = erf(z)/z  (in s = z^2/ZMAX^2)
 *   X(z) = exp(z^2) erfc(z)                                              (in t = z/ZMAX)
 * on 0 <= z <= ZMAX (relative errors below are measured against mpmath).
 */
#pragma once
#define NB_EW_ZMAX 4.0f
/* H: degrees (6,5); fp64 max rel err 6.29e-08; fp32 Horner max rel err 3.47e-07, mean -1.41e-08 */
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
/* E: degrees (5,5); fp64 max rel err 2.48e-08; fp32 Horner max rel err 3.52e-07, mean -1.23e-08 */
#define NB_EW_EP0 1.1283791065216064f
#define NB_EW_EP1 3.096602201461792f
#define NB_EW_EP2 13.59368896484375f
#define NB_EW_EP3 15.904327392578125f
#define NB_EW_EP4 18.647218704223633f
#define NB_EW_EP5 2.0830705165863037f
#define NB_EW_EQ1 8.07761287689209f
#define NB_EW_EQ2 29.528717041015625f
#define NB_EW_EQ3 62.285369873046875f
#define NB_EW_EQ4 77.6876449584961f
#define NB_EW_EQ5 39.23380661010742f
/* X: degrees (4,4); fp64 max rel err 1.1e-08; fp32 Horner max rel err 3.32e-07, mean 7.62e-09 */
#define NB_EW_XP0 1.0f
#define NB_EW_XP1 3.465115547180176f
#define NB_EW_XP2 5.828225612640381f
#define NB_EW_XP3 3.9410693645477295f
#define NB_EW_XP4 0.002993972273543477f
#define NB_EW_XQ1 7.978628158569336f
#define NB_EW_XQ2 25.840158462524414f
#define NB_EW_XQ3 41.050724029541016f
#define NB_EW_XQ4 28.053558349609375f
