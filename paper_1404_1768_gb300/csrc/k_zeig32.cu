// The Schur form of the projected problem (k_zeig.cu) built a second time
// in plain FP32 arithmetic: schur_large_fp32.  It feeds the FP64 Newton
// polish of the warm solve (k_warm.cu) on passes whose pairs are needed
// only to the accuracy that step reaches from an FP32 Schur form -- the
// QR's rotation chains are latency-bound, and FP32 shortens each link.
#define FEAST_QR_FP32 1
#include "k_zeig.cu"
