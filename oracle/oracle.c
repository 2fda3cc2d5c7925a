/*
 * Plain FP64 CPU oracle for the KKT refactor / solve / refine path.
 *
 * TEST INFRASTRUCTURE ONLY. This file is compiled into liboracle.so and is
 * loaded by the test suite, by the smoke check and by the CPU-baseline leg of
 * the benchmark. The product library never links, loads or calls it, and the
 * two share no source, header, table or helper: the only thing they have in
 * common is the seeded problem generator (kktgen), which holds no solver
 * arithmetic.
 *
 * Every routine is written for a reader to check against the paper by eye:
 * no blocking, no fusion, no parallelism, single thread, double precision.
 *
 *   ora_ruiz         equilibration, the first task of the analysis stage
 *                    (Sec. II); reading: symmetric Ruiz iterations rounded to
 *                    powers of 2
 *   ora_min_degree   fill-reducing ordering, part of the analysis stage
 *                    (Sec. II); reading: exact minimum degree on
 *                    the explicit elimination graph, ties to the lowest index
 *   ora_lu           left-looking LU of P*A*Q (Alg. 1: a pivoting LU of the
 *                    first system, then refactorizations of the later ones):
 *                    with p_in == NULL the row order is chosen by threshold
 *                    partial pivoting with diagonal preference; with p_in given
 *                    the pivot sequence is frozen and tiny pivots are replaced
 *                    by static perturbation (reading after Li & Demmel's
 *                    static pivoting)
 *   ora_solve        forward and backward substitution (Alg. 1)
 *   ora_spmv_resid   r = b - K x
 *   ora_backward_error   normwise backward error of x
 *   ora_fgmres       iterative refinement after every solve (Alg. 1; Sec. V
 *                    calls for a better refinement than the library one):
 *                    restarted FGMRES(m), modified Gram-Schmidt, Givens,
 *                    right-preconditioned by the LU solve
 *   ora_lu_error_bound   first-order running error bound of every factor
 *                    entry (Wilkinson), the tolerance of the factor parity
 *
 * Parity is pinned by the tests (dense LAPACK LU, inertia, brute-force fill,
 * closed forms, factors in exact rational arithmetic for the error bound);
 * see tests/test_oracle.py.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ Ruiz */

/* power of two nearest to 1/sqrt(r) in the log2 sense: 2^round(-log2(r)/2) */
static double ora_pow2_inv_sqrt(double r)
{
    int e;
    double m = frexp(r, &e);          /* r = m * 2^e, m in [0.5, 1) */
    /* log2(r) = e + log2(m), log2(m) in [-1, 0) */
    double l2 = (double)e + log2(m);
    double k = -0.5 * l2;
    double kr = floor(k + 0.5);
    return ldexp(1.0, (int)kr);
}

/*
 * Symmetric Ruiz equilibration on a structurally symmetric CSR matrix.
 * d starts at 1; each iteration computes r_i = max_j |d_i a_ij d_j| and sets
 * d_i <- d_i * 2^round(-log2(r_i)/2). Rows with r_i = 0 keep d_i. Stops after
 * `iters` iterations or when an iteration changes no d_i. Returns the number of
 * iterations performed.
 */
int ora_ruiz(int n, const int *rp, const int *ci, const double *v, int iters, double *d)
{
    double *r = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int it;
    for (int i = 0; i < n; i++) d[i] = 1.0;
    for (it = 0; it < iters; it++) {
        int changed = 0;
        for (int i = 0; i < n; i++) {
            double m = 0.0;
            for (int p = rp[i]; p < rp[i + 1]; p++) {
                double a = fabs(d[i] * v[p] * d[ci[p]]);
                if (a > m) m = a;
            }
            r[i] = m;
        }
        for (int i = 0; i < n; i++) {
            if (r[i] > 0.0) {
                double f = ora_pow2_inv_sqrt(r[i]);
                if (f != 1.0) changed = 1;
                d[i] *= f;
            }
        }
        if (!changed) { it++; break; }
    }
    free(r);
    return it;
}

/* ---------------------------------------------------------- min degree */

/*
 * Exact minimum degree on the explicit elimination graph. Adjacency lists are
 * kept as sorted int arrays; eliminating node p makes its uneliminated
 * neighbours a clique. The next node is the uneliminated node of least degree,
 * lowest index first. q[k] receives the node eliminated k-th.
 */
typedef struct { int *a; int n, cap; } ora_set;

static void ora_set_reserve(ora_set *s, int cap)
{
    if (cap > s->cap) {
        int nc = s->cap ? s->cap : 4;
        while (nc < cap) nc *= 2;
        s->a = (int *)realloc(s->a, sizeof(int) * (size_t)nc);
        s->cap = nc;
    }
}

int ora_min_degree(int n, const int *rp, const int *ci, int *q)
{
    ora_set *adj = (ora_set *)calloc((size_t)(n > 0 ? n : 1), sizeof(ora_set));
    char *done = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
    int *tmp = NULL;
    int tmpcap = 0;
    /* degree buckets: doubly linked lists */
    int *head = (int *)malloc(sizeof(int) * (size_t)(n + 1));
    int *next = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int *prev = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int *deg = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i <= n; i++) head[i] = -1;
    for (int i = 0; i < n; i++) {
        ora_set_reserve(&adj[i], rp[i + 1] - rp[i] + 1);
        int c = 0;
        for (int p = rp[i]; p < rp[i + 1]; p++)
            if (ci[p] != i) adj[i].a[c++] = ci[p];
        adj[i].n = c;        /* CSR columns are sorted, so the list is sorted */
        deg[i] = c;
    }
    /* insert in descending index order so each bucket is ascending by index */
    for (int i = n - 1; i >= 0; i--) {
        next[i] = head[deg[i]];
        prev[i] = -1;
        if (head[deg[i]] >= 0) prev[head[deg[i]]] = i;
        head[deg[i]] = i;
    }
    int mindeg = 0;
    for (int k = 0; k < n; k++) {
        while (mindeg <= n && head[mindeg] < 0) mindeg++;
        /* lowest index in the bucket: buckets are not kept sorted after
         * updates, so scan it */
        int p = head[mindeg];
        for (int t = next[p]; t >= 0; t = next[t]) if (t < p) p = t;
        /* unlink p */
        if (prev[p] >= 0) next[prev[p]] = next[p]; else head[deg[p]] = next[p];
        if (next[p] >= 0) prev[next[p]] = prev[p];
        done[p] = 1;
        q[k] = p;
        ora_set *ap = &adj[p];
        /* each neighbour u: adj(u) <- adj(u) U adj(p) minus {u, p} */
        for (int t = 0; t < ap->n; t++) {
            int u = ap->a[t];
            ora_set *au = &adj[u];
            int need = au->n + ap->n;
            if (need > tmpcap) { tmpcap = need * 2; tmp = (int *)realloc(tmp, sizeof(int) * (size_t)tmpcap); }
            int x = 0, y = 0, c = 0;
            while (x < au->n || y < ap->n) {
                int vx = x < au->n ? au->a[x] : 0x7fffffff;
                int vy = y < ap->n ? ap->a[y] : 0x7fffffff;
                int v;
                if (vx < vy) { v = vx; x++; }
                else if (vy < vx) { v = vy; y++; }
                else { v = vx; x++; y++; }
                if (v == u || v == p || done[v]) continue;
                tmp[c++] = v;
            }
            ora_set_reserve(au, c);
            memcpy(au->a, tmp, sizeof(int) * (size_t)c);
            au->n = c;
            /* move u to its new bucket */
            if (prev[u] >= 0) next[prev[u]] = next[u]; else head[deg[u]] = next[u];
            if (next[u] >= 0) prev[next[u]] = prev[u];
            deg[u] = c;
            next[u] = head[c];
            prev[u] = -1;
            if (head[c] >= 0) prev[head[c]] = u;
            head[c] = u;
            if (c < mindeg) mindeg = c;
        }
        free(ap->a);
        ap->a = NULL; ap->n = ap->cap = 0;
    }
    for (int i = 0; i < n; i++) free(adj[i].a);
    free(adj); free(done); free(tmp); free(head); free(next); free(prev); free(deg);
    return 0;
}

/* ------------------------------------------------------------------- LU */

typedef struct {
    int n;
    int *p;        /* p[j]  = original row pivoted at step j            */
    int *q;        /* q[j]  = original column eliminated at step j      */
    int *pinv;     /* pinv[r] = step at which original row r is pivotal */
    /* L: unit lower, CSC over steps; row indices are steps (> column),
     * diagonal not stored. U: upper, CSC over steps; row indices are steps
     * (<= column), ascending, diagonal last. */
    int *Lp, *Li; double *Lx;
    int *Up, *Ui; double *Ux;
    int n_perturbed;
    int n_offdiag;  /* steps whose pivot row differs from the column's own index */
} ora_lu_t;

static void ora_grow_i(int **a, int *cap, int need)
{
    if (need > *cap) {
        int nc = *cap ? *cap : 16;
        while (nc < need) nc *= 2;
        *a = (int *)realloc(*a, sizeof(int) * (size_t)nc);
        *cap = nc;
    }
}
static void ora_grow_d(double **a, int *cap, int need)
{
    if (need > *cap) {
        int nc = *cap ? *cap : 16;
        while (nc < need) nc *= 2;
        *a = (double *)realloc(*a, sizeof(double) * (size_t)nc);
        *cap = nc;
    }
}

static int ora_cmp_int(const void *a, const void *b)
{
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

/*
 * Left-looking (Gilbert-Peierls) LU of P*A*Q.
 *
 * A is given in CSR; its columns are read as the rows of A^T, so the matrix
 * must be structurally symmetric for CSR to double as CSC -- it is (KKT) --
 * but values need not be: column c of A is gathered exactly (A[i][c]) by
 * scanning the CSR rows listed in row c's pattern.
 *
 * Column j (original column q[j]):
 *   x <- A(:, q[j]) over original rows;
 *   for every already-pivotal row r with x_r structurally nonzero, taken in
 *   ascending pivot step k = pinv[r]:  U(k, j) = x_r;  x -= L(:, k) * x_r;
 *   pivot: p_in given -> row p_in[j]; otherwise the column's own row q[j] when
 *   |x_{q[j]}| >= tau * max over candidate rows |x|, else the candidate row
 *   of largest |x| (lowest original index on ties);
 *   static perturbation: |u_jj| < pivot_floor -> u_jj = sign(u_jj) * floor
 *   (sign(0) = +1), counted;
 *   L(:, j) = remaining candidate entries / u_jj.
 * The structural pattern is tracked exactly (entries that cancel to 0.0 are
 * kept), so the pattern equals the symbolic one.
 */
ora_lu_t *ora_lu(int n, const int *rp, const int *ci, const double *v,
                 const int *q, const int *p_in, double tau, double pivot_floor)
{
    ora_lu_t *F = (ora_lu_t *)calloc(1, sizeof(ora_lu_t));
    F->n = n;
    F->p = (int *)malloc(sizeof(int) * (size_t)(n + 1));
    F->q = (int *)malloc(sizeof(int) * (size_t)(n + 1));
    F->pinv = (int *)malloc(sizeof(int) * (size_t)(n + 1));
    F->Lp = (int *)malloc(sizeof(int) * (size_t)(n + 1));
    F->Up = (int *)malloc(sizeof(int) * (size_t)(n + 1));
    int Lcap = 0, Ucap = 0, Lxcap = 0, Uxcap = 0;
    int *Lrow = NULL;   /* L row indices kept as ORIGINAL rows until the end */
    F->Li = NULL; F->Lx = NULL; F->Ui = NULL; F->Ux = NULL;
    memcpy(F->q, q, sizeof(int) * (size_t)n);
    for (int i = 0; i < n; i++) F->pinv[i] = -1;

    double *x = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    char *mark = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
    int *pat = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int *stk = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int *steps = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int lnz = 0, unz = 0;
    F->Lp[0] = 0; F->Up[0] = 0;

    for (int j = 0; j < n; j++) {
        int col = q[j];
        int np = 0;
        /* structural reach of A(:, col) through the columns of L (DFS) */
        for (int t = rp[col]; t < rp[col + 1]; t++) {
            int r0 = ci[t];              /* symmetric pattern: A(r0, col) exists */
            if (mark[r0]) continue;
            int top = 0;
            stk[top++] = r0;
            mark[r0] = 1;
            while (top > 0) {
                int r = stk[--top];
                pat[np++] = r;
                int k = F->pinv[r];
                if (k < 0) continue;
                for (int s = F->Lp[k]; s < F->Lp[k + 1]; s++) {
                    int i = Lrow[s];
                    if (!mark[i]) { mark[i] = 1; stk[top++] = i; }
                }
            }
        }
        /* scatter A(:, col): A(r, col) is stored in row r at column col */
        for (int t = rp[col]; t < rp[col + 1]; t++) {
            int r = ci[t];
            for (int s = rp[r]; s < rp[r + 1]; s++)
                if (ci[s] == col) { x[r] = v[s]; break; }
        }
        /* pivotal rows of the pattern in ascending step order */
        int ns = 0;
        for (int t = 0; t < np; t++) if (F->pinv[pat[t]] >= 0) steps[ns++] = F->pinv[pat[t]];
        qsort(steps, (size_t)ns, sizeof(int), ora_cmp_int);
        ora_grow_i(&F->Ui, &Ucap, unz + ns + 1);
        ora_grow_d(&F->Ux, &Uxcap, unz + ns + 1);
        for (int t = 0; t < ns; t++) {
            int k = steps[t];
            int r = F->p[k];
            double xr = x[r];
            F->Ui[unz] = k; F->Ux[unz] = xr; unz++;
            for (int s = F->Lp[k]; s < F->Lp[k + 1]; s++)
                x[Lrow[s]] -= F->Lx[s] * xr;
        }
        /* choose the pivot among non-pivotal pattern rows */
        int piv = -1;
        if (p_in) {
            piv = p_in[j];
        } else {
            double amax = -1.0;
            int imax = -1;
            int diag_ok = 0;
            for (int t = 0; t < np; t++) {
                int r = pat[t];
                if (F->pinv[r] >= 0) continue;
                double a = fabs(x[r]);
                if (a > amax || (a == amax && r < imax)) { amax = a; imax = r; }
                if (r == col) diag_ok = 1;
            }
            if (diag_ok && fabs(x[col]) >= tau * amax) piv = col;
            else piv = imax >= 0 ? imax : col;
        }
        if (piv != col) F->n_offdiag++;
        double ujj = (piv >= 0 && mark[piv]) ? x[piv] : 0.0;
        if (fabs(ujj) < pivot_floor) {
            ujj = (ujj < 0.0 ? -pivot_floor : pivot_floor);
            F->n_perturbed++;
        }
        F->Ui[unz] = j; F->Ux[unz] = ujj; unz++;
        F->Up[j + 1] = unz;
        F->p[j] = piv;
        F->pinv[piv] = j;
        /* L(:, j): remaining non-pivotal pattern rows, ascending original row */
        int nl = 0;
        for (int t = 0; t < np; t++) {
            int r = pat[t];
            if (F->pinv[r] < 0) stk[nl++] = r;
        }
        qsort(stk, (size_t)nl, sizeof(int), ora_cmp_int);
        ora_grow_i(&Lrow, &Lcap, lnz + nl + 1);
        ora_grow_d(&F->Lx, &Lxcap, lnz + nl + 1);
        for (int t = 0; t < nl; t++) {
            int r = stk[t];
            Lrow[lnz] = r; F->Lx[lnz] = x[r] / ujj; lnz++;
        }
        F->Lp[j + 1] = lnz;
        for (int t = 0; t < np; t++) { x[pat[t]] = 0.0; mark[pat[t]] = 0; }
        if (!mark[piv]) x[piv] = 0.0;
    }
    /* L row indices: original rows -> pivot steps, sorted within each column */
    F->Li = (int *)malloc(sizeof(int) * (size_t)(lnz > 0 ? lnz : 1));
    for (int j = 0; j < n; j++) {
        int a = F->Lp[j], b = F->Lp[j + 1];
        /* pair sort by step: insertion sort on small columns */
        for (int s = a; s < b; s++) F->Li[s] = F->pinv[Lrow[s]];
        for (int s = a + 1; s < b; s++) {
            int ki = F->Li[s]; double kv = F->Lx[s];
            int t = s - 1;
            while (t >= a && F->Li[t] > ki) { F->Li[t + 1] = F->Li[t]; F->Lx[t + 1] = F->Lx[t]; t--; }
            F->Li[t + 1] = ki; F->Lx[t + 1] = kv;
        }
    }
    free(Lrow); free(x); free(mark); free(pat); free(stk); free(steps);
    return F;
}

void ora_lu_free(ora_lu_t *F)
{
    if (!F) return;
    free(F->p); free(F->q); free(F->pinv); free(F->Lp); free(F->Li); free(F->Lx);
    free(F->Up); free(F->Ui); free(F->Ux); free(F);
}

int ora_lu_n(const ora_lu_t *F) { return F->n; }
int ora_lu_nnz_l(const ora_lu_t *F) { return F->Lp[F->n]; }
int ora_lu_nnz_u(const ora_lu_t *F) { return F->Up[F->n]; }
int ora_lu_n_perturbed(const ora_lu_t *F) { return F->n_perturbed; }
int ora_lu_n_offdiag(const ora_lu_t *F) { return F->n_offdiag; }

/* copy out the factors (arrays sized by the counts above) */
void ora_lu_export(const ora_lu_t *F, int *p, int *q, int *Lp, int *Li, double *Lx,
                   int *Up, int *Ui, double *Ux)
{
    int n = F->n;
    memcpy(p, F->p, sizeof(int) * (size_t)n);
    memcpy(q, F->q, sizeof(int) * (size_t)n);
    memcpy(Lp, F->Lp, sizeof(int) * (size_t)(n + 1));
    memcpy(Up, F->Up, sizeof(int) * (size_t)(n + 1));
    memcpy(Li, F->Li, sizeof(int) * (size_t)F->Lp[n]);
    memcpy(Lx, F->Lx, sizeof(double) * (size_t)F->Lp[n]);
    memcpy(Ui, F->Ui, sizeof(int) * (size_t)F->Up[n]);
    memcpy(Ux, F->Ux, sizeof(double) * (size_t)F->Up[n]);
}

/* ---------------------------------------------------------------- solve */

/*
 * Solve (P*A*Q) relation: A z = c  <=>  L U (Q^T z) = P c.
 *   y = L^{-1} c[p]   (forward, unit diagonal, column oriented)
 *   w = U^{-1} y      (backward, column oriented, diagonal stored last)
 *   z[q[j]] = w[j]
 */
void ora_solve(const ora_lu_t *F, const double *c, double *z)
{
    int n = F->n;
    double *y = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int j = 0; j < n; j++) y[j] = c[F->p[j]];
    for (int j = 0; j < n; j++) {
        double yj = y[j];
        for (int s = F->Lp[j]; s < F->Lp[j + 1]; s++) y[F->Li[s]] -= F->Lx[s] * yj;
    }
    for (int j = n - 1; j >= 0; j--) {
        int dpos = F->Up[j + 1] - 1;     /* diagonal is the last entry */
        y[j] /= F->Ux[dpos];
        double yj = y[j];
        for (int s = F->Up[j]; s < dpos; s++) y[F->Ui[s]] -= F->Ux[s] * yj;
    }
    for (int j = 0; j < n; j++) z[F->q[j]] = y[j];
    free(y);
}

/* Scaled solve: K x = b with D K D = A_scaled: x = D * A^{-1} * (D b). */
void ora_solve_scaled(const ora_lu_t *F, const double *d, const double *b, double *x)
{
    int n = F->n;
    double *c = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; i++) c[i] = d[i] * b[i];
    ora_solve(F, c, x);
    for (int i = 0; i < n; i++) x[i] *= d[i];
    free(c);
}

/* ------------------------------------------------------ residual, omega */

void ora_spmv_resid(int n, const int *rp, const int *ci, const double *v,
                    const double *x, const double *b, double *r)
{
    for (int i = 0; i < n; i++) {
        double s = 0.0;
        for (int p = rp[i]; p < rp[i + 1]; p++) s += v[p] * x[ci[p]];
        r[i] = b[i] - s;
    }
}

static double ora_norm_inf(int n, const double *a)
{
    double m = 0.0;
    for (int i = 0; i < n; i++) if (fabs(a[i]) > m) m = fabs(a[i]);
    return m;
}

double ora_matrix_norm_inf(int n, const int *rp, const int *ci, const double *v)
{
    (void)ci;
    double m = 0.0;
    for (int i = 0; i < n; i++) {
        double s = 0.0;
        for (int p = rp[i]; p < rp[i + 1]; p++) s += fabs(v[p]);
        if (s > m) m = s;
    }
    return m;
}

/* omega = ||b - K x||_inf / (||K||_inf ||x||_inf + ||b||_inf) */
double ora_backward_error(int n, const int *rp, const int *ci, const double *v,
                          const double *x, const double *b)
{
    double *r = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    ora_spmv_resid(n, rp, ci, v, x, b, r);
    double num = ora_norm_inf(n, r);
    double den = ora_matrix_norm_inf(n, rp, ci, v) * ora_norm_inf(n, x) + ora_norm_inf(n, b);
    free(r);
    return den > 0.0 ? num / den : num;
}

/* --------------------------------------------------------------- FGMRES */

static double ora_dot(int n, const double *a, const double *b)
{
    double s = 0.0;
    for (int i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

/*
 * Restarted FGMRES(m), right preconditioned by M^{-1} = the scaled LU solve.
 * x0 = M^{-1} b. Each cycle: r = b - K x, beta = ||r||_2, v_1 = r / beta;
 * Arnoldi with modified Gram-Schmidt: z_j = M^{-1} v_j, w = K z_j,
 * h_ij = <w, v_i>, w -= h_ij v_i (i = 1..j), h_{j+1,j} = ||w||, v_{j+1} = w/h;
 * Givens rotations keep the least-squares residual |g_{j+1}|. The inner loop
 * stops when |g_{j+1}| <= tol * (||K||_inf ||x||_inf + ||b||_inf) (a 2-norm
 * bound on the infinity-norm numerator of omega) or j = m; then
 * x += Z y with H y = g solved by back substitution. The true omega is then
 * evaluated; the method stops when omega <= tol or after max_cycles cycles.
 * Returns the number of inner iterations; *omega_out gets the final omega.
 */
int ora_fgmres(int n, const int *rp, const int *ci, const double *v,
               const ora_lu_t *F, const double *d, const double *b, double *x,
               int m, int max_cycles, double tol, double *omega_out)
{
    double *V = (double *)calloc((size_t)n * (size_t)(m + 1), sizeof(double));
    double *Z = (double *)calloc((size_t)n * (size_t)m, sizeof(double));
    double *H = (double *)calloc((size_t)(m + 1) * (size_t)m, sizeof(double));  /* H[i*m + j] */
    double *cs = (double *)calloc((size_t)m, sizeof(double));
    double *sn = (double *)calloc((size_t)m, sizeof(double));
    double *g = (double *)calloc((size_t)(m + 1), sizeof(double));
    double *yv = (double *)calloc((size_t)m, sizeof(double));
    double *w = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *r = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double knorm = ora_matrix_norm_inf(n, rp, ci, v);
    double bnorm = ora_norm_inf(n, b);
    int total = 0;

    ora_solve_scaled(F, d, b, x);
    double omega = ora_backward_error(n, rp, ci, v, x, b);
    for (int cyc = 0; cyc < max_cycles && omega > tol; cyc++) {
        ora_spmv_resid(n, rp, ci, v, x, b, r);
        double beta = sqrt(ora_dot(n, r, r));
        if (beta == 0.0) break;
        double target = tol * (knorm * ora_norm_inf(n, x) + bnorm);
        for (int i = 0; i < n; i++) V[i] = r[i] / beta;
        for (int i = 0; i <= m; i++) g[i] = 0.0;
        g[0] = beta;
        int k = 0;
        for (int j = 0; j < m; j++) {
            double *vj = V + (size_t)j * n, *zj = Z + (size_t)j * n;
            ora_solve_scaled(F, d, vj, zj);
            /* w = K z_j */
            for (int i = 0; i < n; i++) {
                double s = 0.0;
                for (int p = rp[i]; p < rp[i + 1]; p++) s += v[p] * zj[ci[p]];
                w[i] = s;
            }
            for (int i = 0; i <= j; i++) {
                double h = ora_dot(n, w, V + (size_t)i * n);
                H[i * m + j] = h;
                for (int t = 0; t < n; t++) w[t] -= h * V[(size_t)i * n + t];
            }
            double hn = sqrt(ora_dot(n, w, w));
            H[(j + 1) * m + j] = hn;
            if (hn > 0.0)
                for (int t = 0; t < n; t++) V[(size_t)(j + 1) * n + t] = w[t] / hn;
            /* apply previous rotations to column j, then a new one */
            for (int i = 0; i < j; i++) {
                double a = H[i * m + j], c2 = H[(i + 1) * m + j];
                H[i * m + j] = cs[i] * a + sn[i] * c2;
                H[(i + 1) * m + j] = -sn[i] * a + cs[i] * c2;
            }
            double a = H[j * m + j], c2 = H[(j + 1) * m + j];
            double rho = sqrt(a * a + c2 * c2);
            cs[j] = rho > 0.0 ? a / rho : 1.0;
            sn[j] = rho > 0.0 ? c2 / rho : 0.0;
            H[j * m + j] = rho;
            H[(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            k = j + 1;
            total++;
            if (fabs(g[j + 1]) <= target || hn == 0.0) break;
        }
        /* y = H(0:k,0:k)^{-1} g(0:k) */
        for (int i = k - 1; i >= 0; i--) {
            double s = g[i];
            for (int t = i + 1; t < k; t++) s -= H[i * m + t] * yv[t];
            yv[i] = s / H[i * m + i];
        }
        for (int t = 0; t < k; t++)
            for (int i = 0; i < n; i++) x[i] += yv[t] * Z[(size_t)t * n + i];
        omega = ora_backward_error(n, rp, ci, v, x, b);
    }
    if (omega_out) *omega_out = omega;
    free(V); free(Z); free(H); free(cs); free(sn); free(g); free(yv); free(w); free(r);
    return total;
}

/* ------------------------------------------------ running error bounds */

/*
 * First-order running error bound (Wilkinson's running error analysis) for
 * every entry of the factors F of the scaled matrix A (CSR, structurally
 * symmetric), for a computation in a floating-point format of unit roundoff
 * `unit` that forms each entry as in the left-looking elimination of ora_lu
 * in any summation order:
 *
 *   x_i = a_i - sum_k l_ik u_k    (m_i terms)
 *   err(x_i) <= sum_k (|l_ik| err(u_k) + err(l_ik) |u_k|)
 *               + gamma_{m_i+1} (|a_i| + sum_k |l_ik| |u_k|)
 *   u entries: err(u) = err(x);   l_ij = x_i / u_jj, formed either as a
 *   quotient or as x_i * fl(1 / u_jj) (two roundings):
 *   err(l_ij) <= (err(x_i) + |l_ij| err(u_jj)) / |u_jj| + 2 unit |l_ij|
 *
 * gamma_m = m unit / (1 - m unit). A perturbed pivot is the floor rounded
 * once to the format (err unit * pivot_floor; a pivot of magnitude exactly
 * pivot_floor is taken as replaced): FP32 factors hold the FP64 floor rounded
 * to FP32.
 * eL / eU are aligned with Lx / Ux. The bound is first order: it
 * is meaningful only where err(u_jj) < |u_jj| / 2.
 */
void ora_lu_error_bound(const ora_lu_t *F, const int *rp, const int *ci, const double *v,
                        double unit, double pivot_floor, double *eL, double *eU)
{
    int n = F->n;
    double *X = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));   /* |a| + sum |l||u| */
    double *E = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));   /* propagated error */
    int *M = (int *)calloc((size_t)(n > 0 ? n : 1), sizeof(int));
    for (int j = 0; j < n; j++) {
        int col = F->q[j];
        /* |A(:, col)| over original rows */
        for (int t = rp[col]; t < rp[col + 1]; t++) {
            int r = ci[t];
            for (int s = rp[r]; s < rp[r + 1]; s++)
                if (ci[s] == col) { X[r] = fabs(v[s]); break; }
        }
        int dpos = F->Up[j + 1] - 1;
        for (int s = F->Up[j]; s < dpos; s++) {
            int k = F->Ui[s];
            int r = F->p[k];
            double mk = (double)(M[r] + 1);
            double ek = E[r] + (mk * unit / (1.0 - mk * unit)) * X[r];
            eU[s] = ek;
            double uk = fabs(F->Ux[s]);
            for (int t = F->Lp[k]; t < F->Lp[k + 1]; t++) {
                int i = F->p[F->Li[t]];
                double l = fabs(F->Lx[t]);
                E[i] += l * ek + eL[t] * uk;
                X[i] += l * uk;
                M[i] += 1;
            }
        }
        int rj = F->p[j];
        double ujj = F->Ux[dpos];
        double md = (double)(M[rj] + 1);
        double eujj = E[rj] + (md * unit / (1.0 - md * unit)) * X[rj];
        /* replaced pivot: the floor itself, rounded once to the format */
        if (pivot_floor > 0.0 && fabs(ujj) == pivot_floor) eujj = unit * pivot_floor;
        eU[dpos] = eujj;
        double au = fabs(ujj);
        for (int t = F->Lp[j]; t < F->Lp[j + 1]; t++) {
            int i = F->p[F->Li[t]];
            double l = fabs(F->Lx[t]);
            double mi = (double)(M[i] + 1);
            double ex = E[i] + (mi * unit / (1.0 - mi * unit)) * X[i];
            eL[t] = (ex + l * eujj) / au + 2.0 * unit * l;
        }
        /* reset the work arrays on this column's pattern */
        for (int s = F->Up[j]; s <= dpos; s++) { int r = F->p[F->Ui[s]]; X[r] = 0.0; E[r] = 0.0; M[r] = 0; }
        for (int t = F->Lp[j]; t < F->Lp[j + 1]; t++) { int i = F->p[F->Li[t]]; X[i] = 0.0; E[i] = 0.0; M[i] = 0; }
    }
    free(X); free(E); free(M);
}
