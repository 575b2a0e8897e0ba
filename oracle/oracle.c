/*
 * CPU oracle for the PERKS hot path (arXiv 2204.02064).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference legs of bench.py use it.  It shares no code, header, table or
 * helper with the CUDA library; it is plain, slow, serial C written straight
 * from the paper's definitions, in fp64 unless the method fixes another
 * precision.  Build with -O2 -ffp-contract=off so that every a*b+c is two
 * roundings, in the order written.
 *
 * Contents and the passage each function follows:
 *   oracle_stencil_run   Eq. (iterativeStencil), Sec. 2.2.1: Jacobi update,
 *                        every read at step k, written out-of-place; general
 *                        offset/weight table; Dirichlet ghost ring of width r.
 *   oracle_csr_spmv      y = A x for a CSR matrix (the SpMV inside CG,
 *                        Sec. 4.3), row by row, nonzeros in stored order.
 *   oracle_dot           <u, v>, serial left-to-right.
 *   oracle_cg            Conjugate gradient of Sec. 2.2.2 (the commented
 *                        algorithm "Conjugate Gradient Solver"), with the stop
 *                        test read as <r,r> <= (rtol*||b||)^2 and a true-
 *                        residual recomputation on exit (restart if above).
 *   oracle_stencil_run_lowp  The same update with fp32 or bf16 STORAGE (the
 *                        library's low-precision modes): fp32 accumulation
 *                        by fused multiply-add in table order, rounded to the
 *                        storage type after every step.
 *   oracle_bf16_round    float -> bf16 round-to-nearest-even (kept in a float).
 *   oracle_poisson_csr   5-point finite-volume operator of -div(k grad u) on an
 *                        nx*ny grid (h = 1), face coefficient = harmonic mean
 *                        of the two cells' k, Dirichlet 0 through a ghost
 *                        cell with the boundary cell's own k; as CSR.
 *   oracle_conv2d        2-D cross-correlation with zero padding and dilation
 *                        (the warm-start network's layer), fp64.
 *   oracle_warmnet_forward  The 4-layer network: conv+ReLU x3, conv; fp64.
 *   oracle_warmnet_grad  Mean squared error of the network and its gradient
 *                        by reverse-mode chain rule; fp64.
 *   oracle_cg_fp32_ir    Textbook mixed-precision iterative refinement around
 *                        an fp32 CG (not in the paper; the library's FP32-IR
 *                        mode): fp64 residual and correction, fp32 inner CG.
 *
 * Every function here is pinned by tests/test_oracle_*.py against closed
 * forms, invariants and library routines, not against itself.
 *
 * A second build of this same file with -fopenmp (the all-cores CPU
 * baseline of the benchmark, nothing else) runs the planes of each stencil
 * step in parallel; every cell's sum is computed exactly as in the serial
 * build, so the results are identical.
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_ERR_ARG (-1)
#define ORACLE_ERR_NOMEM (-3)
#define ORACLE_NOT_CONVERGED (-7)
#define ORACLE_BREAKDOWN (-8)

/* ------------------------------------------------------------------------ */
/* Stencil                                                                   */
/* ------------------------------------------------------------------------ */

/*
 * Runs `steps` Jacobi steps of y(c) = sum_o w[o] * x(c + off[o]) over the
 * interior of an nx*ny*nz grid (ny = nz = 1 allowed; ndim only checks that
 * offsets stay in the active dimensions).  `off` holds npts (dx,dy,dz)
 * triples, |d| <= radius.  Cells outside the interior read `boundary`
 * (Dirichlet ghost ring of width `radius`).  The sum starts at 0 and adds the
 * terms in table order.  `in` and `out` are interior arrays, x fastest; they
 * may alias.
 */
int oracle_stencil_run(int ndim, int64_t nx, int64_t ny, int64_t nz, int radius,
                       int npts, const int32_t *off, const double *w,
                       double boundary, int64_t steps, const double *in,
                       double *out)
{
    if (ndim < 1 || ndim > 3 || nx < 1 || ny < 1 || nz < 1 || radius < 0 ||
        npts < 1 || steps < 0)
        return ORACLE_ERR_ARG;
    for (int o = 0; o < npts; ++o) {
        for (int d = 0; d < 3; ++d) {
            int v = off[3 * o + d];
            if (v < -radius || v > radius) return ORACLE_ERR_ARG;
            if (d >= ndim && v != 0) return ORACLE_ERR_ARG;
        }
    }
    const int64_t gx = (ndim >= 1) ? radius : 0;
    const int64_t gy = (ndim >= 2) ? radius : 0;
    const int64_t gz = (ndim >= 3) ? radius : 0;
    const int64_t px = nx + 2 * gx, py = ny + 2 * gy, pz = nz + 2 * gz;
    const int64_t total = px * py * pz;
    double *a = (double *)malloc((size_t)total * sizeof(double));
    double *b = (double *)malloc((size_t)total * sizeof(double));
    int64_t *delta = (int64_t *)malloc((size_t)npts * sizeof(int64_t));
    if (!a || !b || !delta) {
        free(a); free(b); free(delta);
        return ORACLE_ERR_NOMEM;
    }
    for (int64_t i = 0; i < total; ++i) { a[i] = boundary; b[i] = boundary; }
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i)
                a[((k + gz) * py + (j + gy)) * px + (i + gx)] =
                    in[(k * ny + j) * nx + i];
    for (int o = 0; o < npts; ++o)
        delta[o] = ((int64_t)off[3 * o + 2] * py + off[3 * o + 1]) * px +
                   off[3 * o + 0];

    for (int64_t s = 0; s < steps; ++s) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
        for (int64_t k = 0; k < nz; ++k)
            for (int64_t j = 0; j < ny; ++j)
                for (int64_t i = 0; i < nx; ++i) {
                    int64_t c = ((k + gz) * py + (j + gy)) * px + (i + gx);
                    double acc = 0.0;
                    for (int o = 0; o < npts; ++o) {
                        double t = w[o] * a[c + delta[o]];
                        acc = acc + t;
                    }
                    b[c] = acc;
                }
        double *t = a; a = b; b = t;
    }
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i)
                out[(k * ny + j) * nx + i] =
                    a[((k + gz) * py + (j + gy)) * px + (i + gx)];
    free(a); free(b); free(delta);
    return ORACLE_OK;
}

/* bf16 keeps the upper 16 bits of an IEEE binary32; rounding to nearest,
 * ties to even, on the discarded 16 bits (finite inputs). */
float oracle_bf16_round(float x)
{
    uint32_t u;
    memcpy(&u, &x, sizeof(u));
    uint32_t lsb = (u >> 16) & 1u;
    u = u + 0x7fffu + lsb;
    u &= 0xffff0000u;
    float y;
    memcpy(&y, &u, sizeof(y));
    return y;
}

/*
 * Low-precision storage variant of oracle_stencil_run: `storage` 1 = fp32,
 * 2 = bf16.  Cells (and the boundary and weights) are held as fp32 values of
 * the storage type; each output is acc = fmaf(w[o], x(c+o), acc) over the
 * table from acc = 0, then rounded to the storage type.  in/out are fp32
 * arrays (bf16 values are exact in fp32).
 */
int oracle_stencil_run_lowp(int ndim, int64_t nx, int64_t ny, int64_t nz, int radius,
                            int npts, const int32_t *off, const double *w,
                            double boundary, int64_t steps, int storage,
                            const float *in, float *out)
{
    if (ndim < 1 || ndim > 3 || nx < 1 || ny < 1 || nz < 1 || radius < 0 ||
        npts < 1 || steps < 0 || (storage != 1 && storage != 2))
        return ORACLE_ERR_ARG;
    for (int o = 0; o < npts; ++o)
        for (int d = 0; d < 3; ++d) {
            int v = off[3 * o + d];
            if (v < -radius || v > radius) return ORACLE_ERR_ARG;
            if (d >= ndim && v != 0) return ORACLE_ERR_ARG;
        }
    const int64_t gx = (ndim >= 1) ? radius : 0;
    const int64_t gy = (ndim >= 2) ? radius : 0;
    const int64_t gz = (ndim >= 3) ? radius : 0;
    const int64_t px = nx + 2 * gx, py = ny + 2 * gy, pz = nz + 2 * gz;
    const int64_t total = px * py * pz;
    float *a = (float *)malloc((size_t)total * sizeof(float));
    float *b = (float *)malloc((size_t)total * sizeof(float));
    int64_t *delta = (int64_t *)malloc((size_t)npts * sizeof(int64_t));
    float *wf = (float *)malloc((size_t)npts * sizeof(float));
    if (!a || !b || !delta || !wf) {
        free(a); free(b); free(delta); free(wf);
        return ORACLE_ERR_NOMEM;
    }
    float bnd = (float)boundary;
    if (storage == 2) bnd = oracle_bf16_round(bnd);
    for (int64_t i = 0; i < total; ++i) { a[i] = bnd; b[i] = bnd; }
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i)
                a[((k + gz) * py + (j + gy)) * px + (i + gx)] = in[(k * ny + j) * nx + i];
    for (int o = 0; o < npts; ++o) {
        delta[o] = ((int64_t)off[3 * o + 2] * py + off[3 * o + 1]) * px + off[3 * o + 0];
        wf[o] = (float)w[o];
    }
    for (int64_t s = 0; s < steps; ++s) {
        for (int64_t k = 0; k < nz; ++k)
            for (int64_t j = 0; j < ny; ++j)
                for (int64_t i = 0; i < nx; ++i) {
                    int64_t c = ((k + gz) * py + (j + gy)) * px + (i + gx);
                    float acc = 0.0f;
                    for (int o = 0; o < npts; ++o) acc = fmaf(wf[o], a[c + delta[o]], acc);
                    b[c] = storage == 2 ? oracle_bf16_round(acc) : acc;
                }
        float *t = a; a = b; b = t;
    }
    for (int64_t k = 0; k < nz; ++k)
        for (int64_t j = 0; j < ny; ++j)
            for (int64_t i = 0; i < nx; ++i)
                out[(k * ny + j) * nx + i] = a[((k + gz) * py + (j + gy)) * px + (i + gx)];
    free(a); free(b); free(delta); free(wf);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Variable-coefficient Poisson operator and the warm-start network           */
/* ------------------------------------------------------------------------ */

static double harmonic(double a, double b) { return 2.0 * a * b / (a + b); }

/* Writes the CSR matrix (rowptr: nx*ny+1, col/val: up to 5*nx*ny) of
 * (Au)_c = sum over the 4 faces of c of kf * (u_c - u_nb), u_nb = 0 outside;
 * kf = harmonic mean of k_c and k_nb inside, k_c on the boundary.  Cell (i,j)
 * is row j*nx + i; columns ascend within a row.  Returns nnz. */
int64_t oracle_poisson_csr(int32_t nx, int32_t ny, const double *k, int32_t *rowptr,
                           int32_t *col, double *val)
{
    int64_t nz = 0;
    rowptr[0] = 0;
    for (int32_t j = 0; j < ny; ++j)
        for (int32_t i = 0; i < nx; ++i) {
            const int32_t c = j * nx + i;
            const double kc = k[c];
            const double fs = j > 0 ? harmonic(kc, k[c - nx]) : kc;
            const double fw = i > 0 ? harmonic(kc, k[c - 1]) : kc;
            const double fe = i + 1 < nx ? harmonic(kc, k[c + 1]) : kc;
            const double fn = j + 1 < ny ? harmonic(kc, k[c + nx]) : kc;
            if (j > 0) { col[nz] = c - nx; val[nz] = -fs; ++nz; }
            if (i > 0) { col[nz] = c - 1; val[nz] = -fw; ++nz; }
            double d = fs + fw;
            d = d + fe;
            d = d + fn;
            col[nz] = c; val[nz] = d; ++nz;
            if (i + 1 < nx) { col[nz] = c + 1; val[nz] = -fe; ++nz; }
            if (j + 1 < ny) { col[nz] = c + nx; val[nz] = -fn; ++nz; }
            rowptr[c + 1] = (int32_t)nz;
        }
    return nz;
}

/* out[co][y][x] = b[co] + sum_ci sum_ky sum_kx w[co][ci][ky][kx] *
 *                 in[ci][y + (ky-1)*dil][x + (kx-1)*dil], zero outside. */
void oracle_conv2d(int32_t cin, int32_t cout, int32_t h, int32_t w, int32_t dil,
                   const double *in, const double *wt, const double *bias, double *out)
{
    for (int32_t co = 0; co < cout; ++co)
        for (int32_t y = 0; y < h; ++y)
            for (int32_t x = 0; x < w; ++x) {
                double acc = bias ? bias[co] : 0.0;
                for (int32_t ci = 0; ci < cin; ++ci)
                    for (int32_t ky = 0; ky < 3; ++ky)
                        for (int32_t kx = 0; kx < 3; ++kx) {
                            const int32_t yy = y + (ky - 1) * dil, xx = x + (kx - 1) * dil;
                            if (yy < 0 || yy >= h || xx < 0 || xx >= w) continue;
                            double t = wt[((co * cin + ci) * 3 + ky) * 3 + kx] *
                                       in[((int64_t)ci * h + yy) * w + xx];
                            acc = acc + t;
                        }
                out[((int64_t)co * h + y) * w + x] = acc;
            }
}

/* Network: channels c0 -> c1 -> c1 -> c1 -> 1, dilations dil[0..3], ReLU
 * after the first three layers.  params holds, per layer, the weights
 * [cout][cin][3][3] followed by the biases [cout].  out: h*w. */
int oracle_warmnet_forward(int32_t c0, int32_t c1, int32_t h, int32_t w, const int32_t *dil,
                           const double *params, const double *in, double *out)
{
    const int32_t cins[4] = {c0, c1, c1, c1}, couts[4] = {c1, c1, c1, 1};
    double *a = (double *)malloc((size_t)c1 * h * w * sizeof(double));
    double *b = (double *)malloc((size_t)c1 * h * w * sizeof(double));
    if (!a || !b) { free(a); free(b); return ORACLE_ERR_NOMEM; }
    const double *x = in;
    const double *p = params;
    for (int l = 0; l < 4; ++l) {
        double *y = (l == 3) ? out : ((l % 2 == 0) ? a : b);
        const double *wt = p;
        const double *bias = p + (int64_t)couts[l] * cins[l] * 9;
        oracle_conv2d(cins[l], couts[l], h, w, dil[l], x, wt, bias, y);
        if (l < 3)
            for (int64_t i = 0; i < (int64_t)couts[l] * h * w; ++i) y[i] = y[i] > 0.0 ? y[i] : 0.0;
        p = bias + couts[l];
        x = y;
    }
    free(a); free(b);
    return ORACLE_OK;
}

/* Mean squared error of the network over nimg images and its gradient with
 * respect to every parameter, by the chain rule written out layer by layer
 * (reverse-mode differentiation of the forward pass above):
 *   L = (1/N) sum (out - t)^2,  N = nimg*h*w,   dL/dout = 2 (out - t) / N;
 *   for a layer y = conv(x; W, b):  dL/db[co] = sum_p dy[co][p],
 *     dL/dW[co][ci][ky][kx] = sum_p dy[co][p] * x[ci][p + off(ky,kx)],
 *     dL/dx[ci][q] = sum_co sum_(ky,kx) W[co][ci][ky][kx] * dy[co][q - off(ky,kx)];
 *   through a ReLU: dL/dz = dL/dy where y = max(z, 0) > 0, else 0.
 * in: nimg*c0*h*w, t: nimg*h*w, grad: same layout as params (overwritten).
 * Returns the loss through *loss. */
int oracle_warmnet_grad(int32_t nimg, int32_t c0, int32_t c1, int32_t h, int32_t w, const int32_t *dil,
                        const double *params, const double *in, const double *t, double *loss, double *grad)
{
    const int32_t cins[4] = {c0, c1, c1, c1}, couts[4] = {c1, c1, c1, 1};
    const int64_t hw = (int64_t)h * w, N = (int64_t)nimg * hw;
    int64_t woff[4], boff[4], np = 0;
    for (int l = 0; l < 4; ++l) {
        woff[l] = np; np += (int64_t)couts[l] * cins[l] * 9;
        boff[l] = np; np += couts[l];
    }
    for (int64_t i = 0; i < np; ++i) grad[i] = 0.0;
    double *act[5];          /* act[0] = input, act[l+1] = output of layer l (after ReLU) */
    double *dy = (double *)malloc((size_t)c1 * hw * sizeof(double));
    double *dx = (double *)malloc((size_t)c1 * hw * sizeof(double));
    int ok = dy && dx;
    for (int l = 1; l <= 4; ++l) {
        act[l] = (double *)malloc((size_t)couts[l - 1] * hw * sizeof(double));
        ok = ok && act[l];
    }
    if (!ok) {
        free(dy); free(dx);
        for (int l = 1; l <= 4; ++l) free(act[l]);
        return ORACLE_ERR_NOMEM;
    }
    double L = 0.0;
    for (int32_t img = 0; img < nimg; ++img) {
        act[0] = (double *)(in + (int64_t)img * c0 * hw);
        for (int l = 0; l < 4; ++l) {
            oracle_conv2d(cins[l], couts[l], h, w, dil[l], act[l], params + woff[l], params + boff[l], act[l + 1]);
            if (l < 3)
                for (int64_t i = 0; i < (int64_t)couts[l] * hw; ++i)
                    act[l + 1][i] = act[l + 1][i] > 0.0 ? act[l + 1][i] : 0.0;
        }
        const double *ti = t + (int64_t)img * hw;
        for (int64_t p = 0; p < hw; ++p) {
            const double d = act[4][p] - ti[p];
            L = L + d * d / (double)N;
            dy[p] = 2.0 * d / (double)N;
        }
        for (int l = 3; l >= 0; --l) {
            const int32_t ci_n = cins[l], co_n = couts[l], d = dil[l];
            const double *x = act[l];
            const double *W = params + woff[l];
            double *gW = grad + woff[l], *gb = grad + boff[l];
            for (int32_t co = 0; co < co_n; ++co)
                for (int64_t p = 0; p < hw; ++p) gb[co] = gb[co] + dy[co * hw + p];
            for (int32_t co = 0; co < co_n; ++co)
                for (int32_t ci = 0; ci < ci_n; ++ci)
                    for (int32_t ky = 0; ky < 3; ++ky)
                        for (int32_t kx = 0; kx < 3; ++kx) {
                            double acc = 0.0;
                            for (int32_t y = 0; y < h; ++y)
                                for (int32_t xq = 0; xq < w; ++xq) {
                                    const int32_t yy = y + (ky - 1) * d, xx = xq + (kx - 1) * d;
                                    if (yy < 0 || yy >= h || xx < 0 || xx >= w) continue;
                                    acc = acc + dy[co * hw + (int64_t)y * w + xq] * x[ci * hw + (int64_t)yy * w + xx];
                                }
                            double *g = &gW[((co * ci_n + ci) * 3 + ky) * 3 + kx];
                            *g = *g + acc;
                        }
            if (l == 0) break;
            for (int64_t i = 0; i < (int64_t)ci_n * hw; ++i) dx[i] = 0.0;
            for (int32_t co = 0; co < co_n; ++co)
                for (int32_t ci = 0; ci < ci_n; ++ci)
                    for (int32_t ky = 0; ky < 3; ++ky)
                        for (int32_t kx = 0; kx < 3; ++kx) {
                            const double wv = W[((co * ci_n + ci) * 3 + ky) * 3 + kx];
                            for (int32_t y = 0; y < h; ++y)
                                for (int32_t xq = 0; xq < w; ++xq) {
                                    const int32_t yy = y + (ky - 1) * d, xx = xq + (kx - 1) * d;
                                    if (yy < 0 || yy >= h || xx < 0 || xx >= w) continue;
                                    double *g = &dx[ci * hw + (int64_t)yy * w + xx];
                                    *g = *g + wv * dy[co * hw + (int64_t)y * w + xq];
                                }
                        }
            /* ReLU of layer l-1: its output is x = act[l] */
            for (int64_t i = 0; i < (int64_t)ci_n * hw; ++i) dy[i] = x[i] > 0.0 ? dx[i] : 0.0;
        }
    }
    *loss = L;
    free(dy); free(dx);
    for (int l = 1; l <= 4; ++l) free(act[l]);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Sparse linear algebra                                                     */
/* ------------------------------------------------------------------------ */

void oracle_csr_spmv(int32_t n, const int32_t *rowptr, const int32_t *col,
                     const double *val, const double *x, double *y)
{
    for (int32_t i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int32_t j = rowptr[i]; j < rowptr[i + 1]; ++j) {
            double t = val[j] * x[col[j]];
            acc = acc + t;
        }
        y[i] = acc;
    }
}

double oracle_dot(int32_t n, const double *u, const double *v)
{
    double acc = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        double t = u[i] * v[i];
        acc = acc + t;
    }
    return acc;
}

/* r = b - A x, returns <r,r>. */
static double residual(int32_t n, const int32_t *rowptr, const int32_t *col,
                       const double *val, const double *b, const double *x,
                       double *r)
{
    oracle_csr_spmv(n, rowptr, col, val, x, r);
    for (int32_t i = 0; i < n; ++i) r[i] = b[i] - r[i];
    return oracle_dot(n, r, r);
}

/*
 * Conjugate gradient, Sec. 2.2.2.  x holds x0 on entry (zeros give the
 * paper's x0 = 0, r0 = b, p0 = b) and the solution on exit.  Per iteration k:
 *   q = A p;  alpha = <r,r>/<p,q>;  x += alpha p;  r -= alpha q;
 *   beta = <r',r'>/<r,r>;  p = r' + beta p;  stop when <r',r'> <= (rtol ||b||)^2.
 * On a stop the true residual b - A x is recomputed in fp64; if it is still
 * above rtol ||b||, CG restarts from the current x (up to max_restarts
 * times).  `iters_out` counts SpMVs of the recurrence (all restarts).
 * `trace`, if not NULL, receives (alpha_k, beta_k, <r_{k+1},r_{k+1}>) for
 * the first trace_len iterations.  Returns 0, NOT_CONVERGED or BREAKDOWN
 * (<p,Ap> <= 0 or not finite).
 */
int oracle_cg(int32_t n, const int32_t *rowptr, const int32_t *col,
              const double *val, const double *b, double *x, double rtol,
              int32_t max_iter, int32_t max_restarts, int32_t *iters_out,
              double *true_rel_out, double *trace, int32_t trace_len)
{
    if (n < 1 || rtol < 0 || max_iter < 0) return ORACLE_ERR_ARG;
    double *r = (double *)malloc((size_t)n * sizeof(double));
    double *p = (double *)malloc((size_t)n * sizeof(double));
    double *q = (double *)malloc((size_t)n * sizeof(double));
    if (!r || !p || !q) { free(r); free(p); free(q); return ORACLE_ERR_NOMEM; }

    const double bb = oracle_dot(n, b, b);
    const double tol2 = rtol * rtol * bb;
    int status = ORACLE_NOT_CONVERGED;
    int32_t it = 0;
    double rr = residual(n, rowptr, col, val, b, x, r);
    for (int32_t restart = 0; restart <= max_restarts; ++restart) {
        if (rr <= tol2) { status = ORACLE_OK; break; }
        memcpy(p, r, (size_t)n * sizeof(double));
        int converged = 0;
        while (it < max_iter) {
            oracle_csr_spmv(n, rowptr, col, val, p, q);
            double pq = oracle_dot(n, p, q);
            if (!(pq > 0.0) || !isfinite(pq)) { status = ORACLE_BREAKDOWN; goto done; }
            double alpha = rr / pq;
            for (int32_t i = 0; i < n; ++i) {
                double t = alpha * p[i];
                x[i] = x[i] + t;
            }
            for (int32_t i = 0; i < n; ++i) {
                double t = alpha * q[i];
                r[i] = r[i] - t;
            }
            double rr_new = oracle_dot(n, r, r);
            double beta = rr_new / rr;
            for (int32_t i = 0; i < n; ++i) {
                double t = beta * p[i];
                p[i] = r[i] + t;
            }
            if (trace && it < trace_len) {
                trace[3 * it + 0] = alpha;
                trace[3 * it + 1] = beta;
                trace[3 * it + 2] = rr_new;
            }
            rr = rr_new;
            ++it;
            if (rr <= tol2) { converged = 1; break; }
        }
        /* C5: true residual in fp64; restart from x if it is above tol. */
        rr = residual(n, rowptr, col, val, b, x, r);
        if (rr <= tol2) { status = ORACLE_OK; break; }
        if (!converged) break; /* out of iterations */
    }
done:
    if (iters_out) *iters_out = it;
    if (true_rel_out) {
        double tr = residual(n, rowptr, col, val, b, x, q);
        *true_rel_out = (bb > 0.0) ? sqrt(tr / bb) : sqrt(tr);
    }
    free(r); free(p); free(q);
    return status;
}

/*
 * Mixed-precision CG: outer iterative refinement in fp64, inner CG in fp32
 * (not in the paper; the library's FP32-IR mode).  Outer step:
 *   r = b - A x (fp64);  stop if ||r|| <= rtol ||b||;
 *   solve A32 d = r32 by fp32 CG from d = 0 until its recurrence residual
 *   <= inner_rtol ||r32|| (or max_inner iterations);  x += d (fp64).
 * A32 and all inner vectors are fp32 and every inner axpy rounds to fp32;
 * the inner dot products accumulate in fp64 (serially) and their results
 * (alpha, beta) are rounded to fp32 before use.
 * `inner_total` receives the number of inner iterations summed over outer
 * steps, `outer_out` the number of outer corrections applied.
 */
int oracle_cg_fp32_ir(int32_t n, const int32_t *rowptr, const int32_t *col,
                      const double *val, const double *b, double *x,
                      double rtol, double inner_rtol, int32_t max_inner,
                      int32_t max_outer, int32_t *inner_total,
                      int32_t *outer_out, double *true_rel_out)
{
    if (n < 1 || rtol < 0 || max_inner < 1 || max_outer < 0) return ORACLE_ERR_ARG;
    const int32_t nnz = rowptr[n];
    double *r = (double *)malloc((size_t)n * sizeof(double));
    float *val32 = (float *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(float));
    float *rf = (float *)malloc((size_t)n * sizeof(float));
    float *pf = (float *)malloc((size_t)n * sizeof(float));
    float *qf = (float *)malloc((size_t)n * sizeof(float));
    float *df = (float *)malloc((size_t)n * sizeof(float));
    if (!r || !val32 || !rf || !pf || !qf || !df) {
        free(r); free(val32); free(rf); free(pf); free(qf); free(df);
        return ORACLE_ERR_NOMEM;
    }
    for (int32_t j = 0; j < nnz; ++j) val32[j] = (float)val[j];
    const double bb = oracle_dot(n, b, b);
    const double tol2 = rtol * rtol * bb;
    int status = ORACLE_NOT_CONVERGED;
    int32_t inner = 0, outer = 0;
    for (;;) {
        double rr64 = residual(n, rowptr, col, val, b, x, r);
        if (rr64 <= tol2) { status = ORACLE_OK; break; }
        if (outer >= max_outer) break;
        /* inner fp32 CG on A32 d = r32, d0 = 0 */
        for (int32_t i = 0; i < n; ++i) {
            rf[i] = (float)r[i]; pf[i] = rf[i]; df[i] = 0.0f;
        }
        double rr = 0.0;
        for (int32_t i = 0; i < n; ++i) rr = rr + (double)rf[i] * (double)rf[i];
        const double itol2 = inner_rtol * inner_rtol * rr;
        for (int32_t k = 0; k < max_inner; ++k) {
            for (int32_t i = 0; i < n; ++i) {
                float acc = 0.0f;
                for (int32_t j = rowptr[i]; j < rowptr[i + 1]; ++j) {
                    float t = val32[j] * pf[col[j]];
                    acc = acc + t;
                }
                qf[i] = acc;
            }
            double pq = 0.0;
            for (int32_t i = 0; i < n; ++i) pq = pq + (double)pf[i] * (double)qf[i];
            if (!(pq > 0.0) || !isfinite(pq)) { status = ORACLE_BREAKDOWN; goto done; }
            float alpha = (float)(rr / pq);
            for (int32_t i = 0; i < n; ++i) {
                float t = alpha * pf[i];
                df[i] = df[i] + t;
            }
            for (int32_t i = 0; i < n; ++i) {
                float t = alpha * qf[i];
                rf[i] = rf[i] - t;
            }
            double rr_new = 0.0;
            for (int32_t i = 0; i < n; ++i) rr_new = rr_new + (double)rf[i] * (double)rf[i];
            float beta = (float)(rr_new / rr);
            for (int32_t i = 0; i < n; ++i) {
                float t = beta * pf[i];
                pf[i] = rf[i] + t;
            }
            rr = rr_new;
            ++inner;
            if (rr <= itol2) break;
        }
        for (int32_t i = 0; i < n; ++i) x[i] = x[i] + (double)df[i];
        ++outer;
    }
done:
    if (inner_total) *inner_total = inner;
    if (outer_out) *outer_out = outer;
    if (true_rel_out) {
        double tr = residual(n, rowptr, col, val, b, x, r);
        *true_rel_out = (bb > 0.0) ? sqrt(tr / bb) : sqrt(tr);
    }
    free(r); free(val32); free(rf); free(pf); free(qf); free(df);
    return status;
}

/* Threads the stencil's parallel loop uses (1 in the serial build). */
int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
