/*
 * FP64 CPU oracle for the dense state-vector simulator (plain C99).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load this file's library. It shares no code,
 * header, table or helper with the CUDA library.
 *
 * What it computes, and where each piece comes from:
 *   - gate application one gate at a time by the flat loop of Algorithm 1
 *     (single target, visit i with the target bit clear, update the pair
 *     (i, i + mask_k) by Eq. 3) and Algorithm 2 (skip indices whose control
 *     bit is clear, Eq. 4); two-target gates update the four amplitudes of
 *     Eq. 6 with local bit 0 = the first target. Controls may sit above or
 *     below the target (the reading of Eq. 4 for any c, t).
 *   - the brute-force unitary: every gate expanded to 2^n x 2^n by Eq. 2
 *     (I (x) ... (x) U (x) ... (x) I, qubit q = bit q), controlled gates as
 *     |0><0| (x) I + |1><1| (x) U (Section 2.1), multiplied in program order.
 *   - Pauli-sum expectation <psi|H|psi> and H|psi> from the textbook action
 *     P|i> = i^{#Y} (-1)^{popcount(i & z)} |i xor x> (Y = iXZ).
 *   - the adjoint gradient of Jones and Gacon (arXiv:2009.02823, Alg. 1).
 * Gate definitions: rotations R_P(a) = exp(-i a P / 2), P(a) = diag(1, e^{ia}),
 * S = diag(1, i), T = diag(1, e^{i pi/4}), H = (X + Z)/sqrt 2.
 *
 * Parity pins: the brute-force unitary (n <= 8), gate identities against
 * scipy's matrix exponential, GHZ and QFT closed forms, circuit * inverse =
 * identity, norm preservation, basis-state Pauli values, and three-way
 * gradient agreement (adjoint, parameter shift, finite differences).
 */
#include "oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/* Threads for the gate loops (the CPU-baseline timing on all host cores):
 * each iteration updates its own pair or quad of amplitudes, so any thread
 * count gives identical results. One thread unless or_set_threads asks. */
#ifdef _OPENMP
#include <omp.h>
#endif
static int g_threads = 1;

int or_set_threads(int t) {
#ifdef _OPENMP
  g_threads = t > 0 ? t : omp_get_num_procs();
#else
  (void)t;
  g_threads = 1;
#endif
  return g_threads;
}

static int popcount64(uint64_t v) {
  int c = 0;
  while (v) { v &= v - 1; ++c; }
  return c;
}

static double gate_angle(const or_gate *g, const double *theta) {
  double a = g->angle;
  if (g->param_index >= 0) a += g->scale * theta[g->param_index];
  return a;
}

static int is_parametric(int kind) {
  return kind == OR_RX || kind == OR_RY || kind == OR_RZ || kind == OR_P;
}

/* Target matrix (row-major). 2x2 for single-target kinds, 4x4 for two-target. */
static int target_matrix(const or_gate *g, const double *theta, cplx *m) {
  const double r2 = 1.0 / sqrt(2.0);
  double a = gate_angle(g, theta);
  double c = cos(0.5 * a), s = sin(0.5 * a);
  switch (g->kind) {
    case OR_H:   m[0] = r2; m[1] = r2; m[2] = r2; m[3] = -r2; return 2;
    case OR_X:   m[0] = 0; m[1] = 1; m[2] = 1; m[3] = 0; return 2;
    case OR_Y:   m[0] = 0; m[1] = -I; m[2] = I; m[3] = 0; return 2;
    case OR_Z:   m[0] = 1; m[1] = 0; m[2] = 0; m[3] = -1; return 2;
    case OR_S:   m[0] = 1; m[1] = 0; m[2] = 0; m[3] = I; return 2;
    case OR_SDG: m[0] = 1; m[1] = 0; m[2] = 0; m[3] = -I; return 2;
    case OR_T:   m[0] = 1; m[1] = 0; m[2] = 0; m[3] = cexp(I * M_PI / 4); return 2;
    case OR_TDG: m[0] = 1; m[1] = 0; m[2] = 0; m[3] = cexp(-I * M_PI / 4); return 2;
    case OR_RX:  m[0] = c; m[1] = -I * s; m[2] = -I * s; m[3] = c; return 2;
    case OR_RY:  m[0] = c; m[1] = -s; m[2] = s; m[3] = c; return 2;
    case OR_RZ:  m[0] = cexp(-0.5 * I * a); m[1] = 0; m[2] = 0; m[3] = cexp(0.5 * I * a); return 2;
    case OR_P:   m[0] = 1; m[1] = 0; m[2] = 0; m[3] = cexp(I * a); return 2;
    case OR_U1:
      for (int k = 0; k < 4; ++k) m[k] = g->mat[2 * k] + I * g->mat[2 * k + 1];
      return 2;
    case OR_SWAP:
      for (int k = 0; k < 16; ++k) m[k] = 0;
      m[0] = 1; m[1 * 4 + 2] = 1; m[2 * 4 + 1] = 1; m[15] = 1;
      return 4;
    case OR_U2:
      for (int k = 0; k < 16; ++k) m[k] = g->mat[2 * k] + I * g->mat[2 * k + 1];
      return 4;
    default: return 0;
  }
}

/* Derivative of the target matrix with respect to the gate's angle. */
static int target_dmatrix(const or_gate *g, const double *theta, cplx *m) {
  double a = gate_angle(g, theta);
  double c = cos(0.5 * a), s = sin(0.5 * a);
  switch (g->kind) {
    case OR_RX: m[0] = -0.5 * s; m[1] = -0.5 * I * c; m[2] = -0.5 * I * c; m[3] = -0.5 * s; return 2;
    case OR_RY: m[0] = -0.5 * s; m[1] = -0.5 * c; m[2] = 0.5 * c; m[3] = -0.5 * s; return 2;
    case OR_RZ: m[0] = -0.5 * I * cexp(-0.5 * I * a); m[1] = 0; m[2] = 0;
                m[3] = 0.5 * I * cexp(0.5 * I * a); return 2;
    case OR_P:  m[0] = 0; m[1] = 0; m[2] = 0; m[3] = I * cexp(I * a); return 2;
    default: return 0;
  }
}

int or_gate_matrix(const or_gate *g, const double *theta, double *m) {
  return target_matrix(g, theta, (cplx *)m);
}

int or_gate_dmatrix(const or_gate *g, const double *theta, double *m) {
  return target_dmatrix(g, theta, (cplx *)m);
}

static uint64_t control_mask(const or_gate *g) {
  uint64_t cm = 0;
  for (int k = 0; k < g->nctrl; ++k) cm |= 1ull << g->ctrl[k];
  return cm;
}

/* Algorithm 1 with the control test of Algorithm 2 in front (Eq. 3, Eq. 4). */
static void apply_single_target(cplx *psi, int n, int t, uint64_t cmask, const cplx *u) {
  const uint64_t mask_t = 1ull << t;
  const uint64_t dim = 1ull << n;
#pragma omp parallel for schedule(static) num_threads(g_threads) if (g_threads > 1)
  for (uint64_t i = 0; i < dim; ++i) {
    if ((i & cmask) != cmask) continue;
    if (i & mask_t) continue;
    cplx a0 = psi[i];
    cplx a1 = psi[i + mask_t];
    psi[i] = u[0] * a0 + u[1] * a1;
    psi[i + mask_t] = u[2] * a0 + u[3] * a1;
  }
}

/* Eq. 6: the four amplitudes (b_t2 b_t1) = 00, 01, 10, 11 with t1 = targ[0]. */
static void apply_two_target(cplx *psi, int n, int t1, int t2, uint64_t cmask, const cplx *u) {
  const uint64_t m1 = 1ull << t1, m2 = 1ull << t2;
  const uint64_t dim = 1ull << n;
#pragma omp parallel for schedule(static) num_threads(g_threads) if (g_threads > 1)
  for (uint64_t i = 0; i < dim; ++i) {
    if ((i & cmask) != cmask) continue;
    if (i & (m1 | m2)) continue;
    uint64_t idx[4] = {i, i | m1, i | m2, i | m1 | m2};
    cplx a[4];
    for (int r = 0; r < 4; ++r) a[r] = psi[idx[r]];
    for (int r = 0; r < 4; ++r) {
      cplx acc = 0;
      for (int c = 0; c < 4; ++c) acc += u[4 * r + c] * a[c];
      psi[idx[r]] = acc;
    }
  }
}

static void apply_matrix(cplx *psi, int n, const or_gate *g, const cplx *u, int d) {
  uint64_t cm = control_mask(g);
  if (d == 2) apply_single_target(psi, n, g->targ[0], cm, u);
  else apply_two_target(psi, n, g->targ[0], g->targ[1], cm, u);
}

void or_set_basis(double *psi, int n, uint64_t x) {
  memset(psi, 0, sizeof(cplx) << n);
  ((cplx *)psi)[x] = 1.0;
}

void or_apply_gate(double *psi, int n, const or_gate *g, const double *theta) {
  cplx u[16];
  int d = target_matrix(g, theta, u);
  apply_matrix((cplx *)psi, n, g, u, d);
}

void or_apply_gate_adjoint(double *psi, int n, const or_gate *g, const double *theta) {
  cplx u[16], ua[16];
  int d = target_matrix(g, theta, u);
  for (int r = 0; r < d; ++r)
    for (int c = 0; c < d; ++c) ua[r * d + c] = conj(u[c * d + r]);
  apply_matrix((cplx *)psi, n, g, ua, d);
}

void or_apply_circuit(double *psi, int n, const or_gate *g, int64_t ng, const double *theta) {
  for (int64_t k = 0; k < ng; ++k) or_apply_gate(psi, n, &g[k], theta);
}

double or_norm2(const double *psi, int n) {
  const cplx *p = (const cplx *)psi;
  double s = 0;
  for (uint64_t i = 0; i < (1ull << n); ++i) s += creal(p[i]) * creal(p[i]) + cimag(p[i]) * cimag(p[i]);
  return s;
}

/* ---------------- brute force (Eq. 2) ---------------- */

/* G += coeff * (m[n-1] (x) ... (x) m[0]); m[q] is the 2x2 factor on qubit q. */
static void kron_chain_add(int n, cplx m[][4], cplx coeff, cplx *G) {
  const uint64_t dim = 1ull << n;
  for (uint64_t r = 0; r < dim; ++r)
    for (uint64_t c = 0; c < dim; ++c) {
      cplx v = coeff;
      for (int q = 0; q < n && v != 0; ++q) v *= m[q][2 * ((r >> q) & 1) + ((c >> q) & 1)];
      G[r * dim + c] += v;
    }
}

static void set_identity_factors(int n, cplx m[][4]) {
  for (int q = 0; q < n; ++q) { m[q][0] = 1; m[q][1] = 0; m[q][2] = 0; m[q][3] = 1; }
}

/* Full 2^n x 2^n matrix of one gate:
 *   G = I - P1(C) + P1(C) (x) U   where P1(C) = product of |1><1| on the controls. */
static void full_gate_matrix(int n, const or_gate *g, const double *theta, cplx *G) {
  const uint64_t dim = 1ull << n;
  cplx u[16];
  int d = target_matrix(g, theta, u);
  cplx (*m)[4] = malloc(sizeof(cplx[4]) * (size_t)n);
  memset(G, 0, sizeof(cplx) * dim * dim);
  if (g->nctrl > 0) {
    set_identity_factors(n, m);
    kron_chain_add(n, m, 1.0, G);
    for (int k = 0; k < g->nctrl; ++k) { int q = g->ctrl[k]; m[q][0] = 0; m[q][3] = 1; }
    kron_chain_add(n, m, -1.0, G);
  }
  if (d == 2) {
    set_identity_factors(n, m);
    for (int k = 0; k < g->nctrl; ++k) { int q = g->ctrl[k]; m[q][0] = 0; m[q][3] = 1; }
    for (int k = 0; k < 4; ++k) m[g->targ[0]][k] = u[k];
    kron_chain_add(n, m, 1.0, G);
  } else {
    /* U = sum over (r2 r1, c2 c1) of U[r,c] E_{r2 c2}(t2) (x) E_{r1 c1}(t1) */
    for (int r = 0; r < 4; ++r)
      for (int c = 0; c < 4; ++c) {
        if (u[4 * r + c] == 0) continue;
        set_identity_factors(n, m);
        for (int k = 0; k < g->nctrl; ++k) { int q = g->ctrl[k]; m[q][0] = 0; m[q][3] = 1; }
        int q1 = g->targ[0], q2 = g->targ[1];
        for (int k = 0; k < 4; ++k) { m[q1][k] = 0; m[q2][k] = 0; }
        m[q1][2 * (r & 1) + (c & 1)] = 1;
        m[q2][2 * (r >> 1) + (c >> 1)] = 1;
        kron_chain_add(n, m, u[4 * r + c], G);
      }
  }
  free(m);
}

void or_unitary(int n, const or_gate *g, int64_t ng, const double *theta, double *Uout) {
  const uint64_t dim = 1ull << n;
  cplx *U = (cplx *)Uout;
  cplx *G = malloc(sizeof(cplx) * dim * dim);
  cplx *T = malloc(sizeof(cplx) * dim * dim);
  memset(U, 0, sizeof(cplx) * dim * dim);
  for (uint64_t i = 0; i < dim; ++i) U[i * dim + i] = 1;
  for (int64_t k = 0; k < ng; ++k) {
    full_gate_matrix(n, &g[k], theta, G);
    for (uint64_t r = 0; r < dim; ++r)           /* T = G U */
      for (uint64_t c = 0; c < dim; ++c) {
        cplx acc = 0;
        for (uint64_t j = 0; j < dim; ++j) acc += G[r * dim + j] * U[j * dim + c];
        T[r * dim + c] = acc;
      }
    memcpy(U, T, sizeof(cplx) * dim * dim);
  }
  free(G);
  free(T);
}

/* ---------------- Pauli sums ---------------- */

static cplx i_pow(int k) {
  switch (k & 3) { case 0: return 1; case 1: return I; case 2: return -1; default: return -I; }
}

double or_expval(const double *psi_, int n, const double *coeff, const uint64_t *xm,
                 const uint64_t *zm, int64_t nt, double *imag_out) {
  const cplx *psi = (const cplx *)psi_;
  const uint64_t dim = 1ull << n;
  cplx total = 0;
  for (int64_t j = 0; j < nt; ++j) {
    cplx s = 0;
    for (uint64_t i = 0; i < dim; ++i) {
      double sign = (popcount64(i & zm[j]) & 1) ? -1.0 : 1.0;
      s += conj(psi[i ^ xm[j]]) * sign * psi[i];
    }
    total += coeff[j] * i_pow(popcount64(xm[j] & zm[j])) * s;
  }
  if (imag_out) *imag_out = cimag(total);
  return creal(total);
}

void or_apply_pauli_sum(const double *psi_, int n, const double *coeff, const uint64_t *xm,
                        const uint64_t *zm, int64_t nt, double *out_) {
  const cplx *psi = (const cplx *)psi_;
  cplx *out = (cplx *)out_;
  const uint64_t dim = 1ull << n;
  memset(out, 0, sizeof(cplx) * dim);
  for (int64_t j = 0; j < nt; ++j) {
    cplx ph = coeff[j] * i_pow(popcount64(xm[j] & zm[j]));
    for (uint64_t i = 0; i < dim; ++i) {
      double sign = (popcount64(i & zm[j]) & 1) ? -1.0 : 1.0;
      out[i ^ xm[j]] += ph * sign * psi[i];
    }
  }
}

/* ---------------- adjoint gradient ---------------- */

/* mu = (d G / d angle) phi: the derivative matrix on the controlled subspace,
 * zero where any control bit is clear. */
static void apply_derivative(const cplx *phi, cplx *mu, int n, const or_gate *g, const cplx *du) {
  const uint64_t dim = 1ull << n;
  const uint64_t cm = control_mask(g);
  const uint64_t mask_t = 1ull << g->targ[0];
  memset(mu, 0, sizeof(cplx) * dim);
  for (uint64_t i = 0; i < dim; ++i) {
    if ((i & cm) != cm) continue;
    if (i & mask_t) continue;
    cplx a0 = phi[i], a1 = phi[i + mask_t];
    mu[i] = du[0] * a0 + du[1] * a1;
    mu[i + mask_t] = du[2] * a0 + du[3] * a1;
  }
}

int or_adjoint_grad(const double *psi0, int n, const or_gate *g, int64_t ng,
                    const double *theta, int64_t ntheta, const double *coeff,
                    const uint64_t *xm, const uint64_t *zm, int64_t nt,
                    double *expval, double *grad) {
  const uint64_t dim = 1ull << n;
  cplx *phi = malloc(sizeof(cplx) * dim);
  cplx *lam = malloc(sizeof(cplx) * dim);
  cplx *mu = malloc(sizeof(cplx) * dim);
  if (!phi || !lam || !mu) { free(phi); free(lam); free(mu); return -1; }
  for (int64_t p = 0; p < ntheta; ++p) grad[p] = 0;
  memcpy(phi, psi0, sizeof(cplx) * dim);
  or_apply_circuit((double *)phi, n, g, ng, theta);
  or_apply_pauli_sum((const double *)phi, n, coeff, xm, zm, nt, (double *)lam);
  cplx e = 0;
  for (uint64_t i = 0; i < dim; ++i) e += conj(phi[i]) * lam[i];
  *expval = creal(e);
  for (int64_t k = ng - 1; k >= 0; --k) {
    or_apply_gate_adjoint((double *)phi, n, &g[k], theta);
    if (g[k].param_index >= 0 && is_parametric(g[k].kind)) {
      cplx du[4];
      target_dmatrix(&g[k], theta, du);
      apply_derivative(phi, mu, n, &g[k], du);
      cplx s = 0;
      for (uint64_t i = 0; i < dim; ++i) s += conj(lam[i]) * mu[i];
      grad[g[k].param_index] += g[k].scale * 2.0 * creal(s);
    }
    or_apply_gate_adjoint((double *)lam, n, &g[k], theta);
  }
  free(phi); free(lam); free(mu);
  return 0;
}
