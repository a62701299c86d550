/*
 * CPU oracle for the parallel in-place merge of
 *   B. Bramas, Q. Bramas, "On the improvement of the in-place merge algorithm
 *   parallelization", arXiv 2005.12648.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is loaded by tests/, by the smoke check in
 * __graft_entry__.py and by the CPU-baseline and reference legs of bench.py, and by
 * nothing else.  The product path (the CUDA library and its Python binding) never
 * links, loads or calls it, and the two share no code: no kernels, headers,
 * helpers, tables or constants.
 *
 * It is deliberately plain, sequential and slow: each function is the definition or
 * the paper's algorithm written out in the paper's order, with no blocking, fusion
 * or reordering.  The typed functions live in oracle_typed.h, included once per key
 * type.  The learned split proposer (a 1 -> H -> 1 tanh MLP trained with Adam) has
 * no counterpart in the paper; its float64 forward, backward and Adam step below are
 * the textbook definitions.
 *
 * Parity unpinned: FindMedian's balance against the optimal split (the E1 comparison
 * of Sec. 4) is given by the paper only as a plot, so orc_findmedian and orc_division
 * with FindMedian pivots are pinned by FindMedian's corner cases and the validity of
 * its splits, not by the paper's values.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#define T int32_t
#define SUF i32
#include "oracle_typed.h"
#undef T
#undef SUF

#define T uint32_t
#define SUF u32
#include "oracle_typed.h"
#undef T
#undef SUF

#define T uint64_t
#define SUF u64
#include "oracle_typed.h"
#undef T
#undef SUF

#define T float
#define SUF f32
#include "oracle_typed.h"
#undef T
#undef SUF

#define T int64_t
#define SUF i64
#include "oracle_typed.h"
#undef T
#undef SUF

/* ------------------------------------------------------------------------------ */
/* Learned split proposer: y(x) = b2 + sum_h w2[h] * tanh(w1[h] * x + b1[h]).       */
/* Parameter layout (3H+1 doubles): w1[0..H), b1[0..H), w2[0..H), b2.               */
/* ------------------------------------------------------------------------------ */

void orc_mlp_forward(const double *prm, int H, const double *x, uint64_t n, double *y)
{
    const double *w1 = prm, *b1 = prm + H, *w2 = prm + 2 * H, b2 = prm[3 * H];
    for (uint64_t s = 0; s < n; ++s) {
        double acc = b2;
        for (int h = 0; h < H; ++h) acc += w2[h] * tanh(w1[h] * x[s] + b1[h]);
        y[s] = acc;
    }
}

/*
 * Mean squared error L = (1/n) sum_s (y(x_s) - t_s)^2 and, when grad is not NULL,
 * its gradient with respect to the 3H+1 parameters (chain rule, d tanh(u)/du =
 * 1 - tanh(u)^2).
 */
double orc_mlp_loss_grad(const double *prm, int H, const double *x, const double *t,
                         uint64_t n, double *grad)
{
    const double *w1 = prm, *b1 = prm + H, *w2 = prm + 2 * H, b2 = prm[3 * H];
    double loss = 0.0;
    if (grad) memset(grad, 0, sizeof(double) * (size_t)(3 * H + 1));
    for (uint64_t s = 0; s < n; ++s) {
        double y = b2;
        for (int h = 0; h < H; ++h) y += w2[h] * tanh(w1[h] * x[s] + b1[h]);
        double r = y - t[s];
        loss += r * r;
        if (grad) {
            double g = 2.0 * r / (double)n; /* dL/dy_s */
            for (int h = 0; h < H; ++h) {
                double a = tanh(w1[h] * x[s] + b1[h]);
                double du = g * w2[h] * (1.0 - a * a);
                grad[h] += du * x[s];       /* w1 */
                grad[H + h] += du;          /* b1 */
                grad[2 * H + h] += g * a;   /* w2 */
            }
            grad[3 * H] += g;               /* b2 */
        }
    }
    return loss / (double)n;
}

/*
 * One Adam step (Kingma & Ba): m <- b1 m + (1-b1) g; v <- b2 v + (1-b2) g^2;
 * p <- p - lr * mhat / (sqrt(vhat) + eps) with mhat = m/(1-b1^step),
 * vhat = v/(1-b2^step); step counts from 1.
 */
void orc_adam_step(double *prm, double *m, double *v, const double *g, int np, double lr,
                   double beta1, double beta2, double eps, int step)
{
    double c1 = 1.0 - pow(beta1, (double)step), c2 = 1.0 - pow(beta2, (double)step);
    for (int q = 0; q < np; ++q) {
        m[q] = beta1 * m[q] + (1.0 - beta1) * g[q];
        v[q] = beta2 * v[q] + (1.0 - beta2) * g[q] * g[q];
        prm[q] -= lr * (m[q] / c1) / (sqrt(v[q] / c2) + eps);
    }
}
