/* pic2d.h -- C ABI of subsystem I of the two-dimensional scheme (libpic, sm_103a).
 *
 * The paper's two-dimensional reduced model (Sec. 2.2) discretised on tensor-
 * product splines (Sec. 3.2) on a uniform periodic M1 x M2 grid: node index
 * i = i1 * M2 + i2; A_z in V0 (basis N^k(x1/dx1 - i1) N^k(x2/dx2 - i2)); the
 * 1-form e_xy in V1 as two component arrays, e_x on N^{k-1} x N^k and e_y on
 * N^k x N^{k-1}.  Markers carry x = (x1, x2) in [0, L1) x [0, L2) and
 * p = (p_x, p_y), equal weights w and, with hbar != 0, spins s = (s_x, s_y, s_z)
 * with the 2-form b_z (N^{k-1} x N^{k-1}).  What is built is subsystem I of the 2D
 * splitting (Sec. 4.3): the discrete-gradient scheme
 *   x^{n+1} - x^n = dt (p^n + p^{n+1}) / (g(p^n, A(x^{n+1})) + g(p^{n+1}, A(x^{n+1}))),
 *   p^{n+1} - p^n = int_{t^n}^{t^{n+1}} Lambda_1^T(x(t)) dt e_bar
 *                   - dt (A(x^{n+1}) + A(x^n)) D / (g(p^n, A(x^{n+1})) + g(p^n, A(x^n)))
 *                   - dt hbar (s_x D[dA/dx2] - s_y D[dA/dx1] + s_z D[b_z]),
 *   e^{n+1} - e^n = -M1^{-1} sum_a w int Lambda_1 . dx along x^n -> x^{n+1},
 * g(p, A) = sqrt(1 + |p|^2 + A^2), e_bar = (e^n + e^{n+1}) / 2, D[f] the
 * coordinate-increment difference quotients of f (along x1 at x2^{n+1}, then
 * along x2 at x1^n), taken as exact path means of the derivatives, and
 * M1 = diag(M1_x (x) M0_y, M0_x (x) M1_y).  The Zeeman term is that of the 2D
 * Hamiltonian (Eq. discrete_H2d), + hbar s . B with B = (dA_z/dx2, -dA_z/dx1, b_z);
 * spins and b_z are constant in this subsystem.  The fixed point is a Picard
 * iteration on the positions (from x^(0) = x^n, or the explicit predictor with
 * its consistent field, see pic2d_config.warm) with one e_xy update per sweep,
 * stopped when the position, momentum and field increments are all at most tol.
 * All arithmetic is FP64.
 *
 * Conventions as in pic.h: return PIC_OK or a PIC_ERR_* code, message via
 * pic2d_last_error(h) (or pic2d_last_error(NULL) after a failed init); the handle
 * owns its device memory; arrays are host (PIC_MEM_HOST) or device
 * (PIC_MEM_DEVICE) pointers, row-major (np x 2) for x and p.  Grids: 1 <= M1, M2,
 * M1 * M2 <= 4096, degree 2..5.
 */
#ifndef PIC2D_H
#define PIC2D_H

#include <stdint.h>

#include "pic.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pic2d_config {
    double L1, L2;       /* domain lengths */
    int32_t M1, M2;      /* cells along x1, x2 */
    int32_t degree;      /* k: A_z in degree k, e_xy components mixed k-1 / k */
    int64_t np;          /* markers */
    double weight;       /* w, equal for every marker */
    double dt;           /* time step */
    double tol;          /* absolute tolerance on the max-norm of the increments */
    int32_t max_iter;    /* sweep cap of the fixed point */
    double hbar;         /* 0: no spin terms; else pic2d_set_spin before the first step */
    int32_t warm;        /* start of the fixed point: 0 = x^(0) = x^n with e^(0) = e^n;
                            1 = the explicit predictor x^(0) = x^n + dt p^n / g(p^n, A(x^n))
                            with the field consistent with it, e^(0) = e^n - M1^{-1} j(x^n -> x^(0))
                            (the same fixed point; fewer sweeps) */
} pic2d_config;

typedef struct pic2d_handle pic2d_handle;

/* Create the state on the current device: x, p (np x 2), e_x, e_y, a_z (M1 * M2).
 * Errors: PIC_ERR_INVALID (configuration, positions outside the box),
 * PIC_ERR_NOMEM, PIC_ERR_CUDA. */
int pic2d_init(const pic2d_config *cfg, const double *x, const double *p, const double *ex,
               const double *ey, const double *az, int32_t mem, void *stream, pic2d_handle **out);

/* Spins s (np x 3, row-major) and b_z (M1 * M2) for the Zeeman terms (hbar != 0);
 * may be called again to replace them.  Errors: PIC_ERR_INVALID (null, b_z not
 * finite), PIC_ERR_NOMEM, PIC_ERR_CUDA. */
int pic2d_set_spin(pic2d_handle *h, const double *s, const double *bz, int32_t mem);

/* One step of subsystem I (Sec. 4.3) by dt; *iters (may be NULL) = sweeps.
 * PIC_ERR_NOCONVERGE: max_iter reached (state = last iterate); PIC_ERR_NUMERIC:
 * non-finite values or a displacement of more than 16 cells; PIC_ERR_INVALID:
 * hbar != 0 and no spins given. */
int pic2d_substep1(pic2d_handle *h, int32_t *iters);

/* out[0] = sum_a w (g(p_a, A(x_a)) - 1), out[1] = e^T M1 e / 2, out[2] = the
 * Zeeman energy hbar sum_a w (s_x dA_z/dx2 - s_y dA_z/dx1 + s_z b_z)(x_a) (0
 * without spins), out[3] = their sum (the part of the discrete Hamiltonian,
 * Eq. discrete_H2d, that subsystem I exchanges; the other terms are constant in it). */
int pic2d_energy(pic2d_handle *h, double out[4]);

/* Copy x, p (np x 2) and e_x, e_y (M1 * M2) out (any may be NULL). */
int pic2d_get_state(pic2d_handle *h, double *x, double *p, double *ex, double *ey, int32_t mem);

int pic2d_destroy(pic2d_handle *h);
const char *pic2d_last_error(const pic2d_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* PIC2D_H */
