/*
 * FP64 CPU oracle for the dense state-vector simulator.
 *
 * TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
 * CPU-baseline leg call it; the CUDA library never includes, links or calls
 * anything here, and nothing here includes the library's headers.
 *
 * Storage: a state of n qubits is 2^n complex doubles (re, im interleaved,
 * C99 `double complex`); qubit q is bit q of the index (Section 2.1, Eq. 1-2).
 * All routines are single-threaded, unblocked and apply one gate at a time.
 */
#ifndef GB300_SV_ORACLE_H
#define GB300_SV_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Gate kinds understood by the oracle (own numbering). */
enum {
  OR_H = 1, OR_X, OR_Y, OR_Z, OR_S, OR_SDG, OR_T, OR_TDG,
  OR_RX, OR_RY, OR_RZ, OR_P, OR_U1, OR_SWAP, OR_U2
};

typedef struct {
  int32_t kind;
  int32_t ntarg;        /* 1 or 2 */
  int32_t targ[2];
  int32_t nctrl;        /* 0..2 */
  int32_t ctrl[2];
  int32_t param_index;  /* -1: fixed angle */
  double angle;         /* angle, or offset when param_index >= 0 */
  double scale;         /* angle += scale * theta[param_index] */
  double mat[32];       /* U1: 2x2, U2: 4x4, row-major (re, im) pairs */
} or_gate;

/* Target matrix of a gate (2x2 or 4x4, row-major complex); returns its size.
 * The U of Eq. 3-4 and Eq. 6: fixed gates by their standard matrices,
 * rotations R_P(a) = exp(-i a P / 2), P(a) = diag(1, e^{ia}). */
int or_gate_matrix(const or_gate *g, const double *theta, double *m);
/* d(target matrix)/d(angle) for parametric kinds; returns 0 for fixed kinds. */
int or_gate_dmatrix(const or_gate *g, const double *theta, double *m);

/* |x> of Eq. 1. */
/* Threads the gate loops use (t <= 0: all processors); returns the count in
 * effect (1 when built without OpenMP). Results do not depend on it. */
int or_set_threads(int t);
void or_set_basis(double *psi, int n, uint64_t x);
/* One gate in place: Algorithm 1 / Eq. 3 (pairs i, i + 2^t) for one target,
 * Algorithm 2 / Eq. 4 (only indices whose control bits are all 1) for
 * controls above or below the target, Eq. 6's quads for two targets. */
void or_apply_gate(double *psi, int n, const or_gate *g, const double *theta);
/* The same with the gate's conjugate transpose (adjoint method, Jones and
 * Gacon 2020). */
void or_apply_gate_adjoint(double *psi, int n, const or_gate *g, const double *theta);
/* psi <- G_N ... G_1 psi, one gate at a time: the plain result the fused
 * method reaches (Section 3.4). */
void or_apply_circuit(double *psi, int n, const or_gate *g, int64_t ng, const double *theta);
/* sum_i |psi_i|^2 (textbook). */
double or_norm2(const double *psi, int n);

/* Brute-force 2^n x 2^n unitary of a circuit from Eq. 2 Kronecker products. */
void or_unitary(int n, const or_gate *g, int64_t ng, const double *theta, double *U);

/* <psi| sum_j c_j P_j |psi>; *imag_out receives the imaginary part. Uses
 * P|i> = i^{#Y} (-1)^{popcount(i & z)} |i xor x> with Y = iXZ (textbook). */
double or_expval(const double *psi, int n, const double *coeff, const uint64_t *xm,
                 const uint64_t *zm, int64_t nt, double *imag_out);
/* out = sum_j c_j P_j psi. */
void or_apply_pauli_sum(const double *psi, int n, const double *coeff, const uint64_t *xm,
                        const uint64_t *zm, int64_t nt, double *out);

/* Adjoint-method gradient (Jones and Gacon 2020, arXiv:2009.02823) of
 * <psi(theta)|H|psi(theta)>, psi(theta) = C(theta) psi0.
 * grad has ntheta entries (zeroed here). Returns 0, or -1 on allocation failure. */
int or_adjoint_grad(const double *psi0, int n, const or_gate *g, int64_t ng,
                    const double *theta, int64_t ntheta, const double *coeff,
                    const uint64_t *xm, const uint64_t *zm, int64_t nt,
                    double *expval, double *grad);

#ifdef __cplusplus
}
#endif
#endif
