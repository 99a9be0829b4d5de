/*
 * cs_oracle.c -- plain, slow, FP64 CPU oracle for cascading-smoother
 * multigrid.  TEST INFRASTRUCTURE ONLY: it is used by tests/, by the smoke
 * check and by the benchmark's CPU-baseline leg, never by the library.  It
 * shares no code, header, table or helper with the CUDA path.
 *
 * Everything here works on general CSR matrices so that each step can be
 * read against the paper:
 *   - additive cascade setup ............ Sec. 2.1 and Algorithm 2
 *   - multiplicative (coloured) setup ... Sec. 2.2 and SM Algorithm
 *     (snapshot per colour, i.e. E_{l,k} = (I - Lambda_{l,k} A) E_{l,k-1})
 *   - elliptic prescaling W = diag(A_ii^{-1/2}) ... Sec. 2.3.1
 *   - forward application eq. (fwda) / (fwdm); reverse application
 *     eq. (fwdar) / (fwdmr) read as Lambda_{nu-l+1}^T (and colour chi-k+1),
 *     the order fixed by the reverse propagator of SM Sec. 3
 *   - V-cycle ......................... Algorithm 1
 *   - Galerkin coarse operator A_2h = R A_h P with R = 2^{-d} P^T (SM 4.1),
 *     or rscale P^T A P for a user CSR hierarchy with user blocks
 *   - coarsest direct solve: Cholesky for a symmetric matrix, LU with
 *     partial pivoting otherwise (Algorithm 1)
 *   - outer solves: stationary, left-preconditioned GMRES (Sec. 3.1), the
 *     same with the cycle on the right (flexible form), and PCG (SM "On
 *     preconditioned conjugate gradient")
 *   - greedy colouring of the block graph in hash-priority order (Sec. 3.4)
 *   - sketched setup min ||(E - Lambda R) S||_F, Rademacher S (Sec. 4)
 *   - Stokes prescaling (Sec. 2.3; SM "Prescaling Stokes problems")
 *   - overlapping blocks with theta-averaged fusion (Sec. 3.6.2) and the
 *     SPD projection of Lambda blocks bounded by block Jacobi (SM, PCG)
 *
 * No blocking, fusion or reordering beyond what those definitions state.
 *
 * Planted mistakes (ora_plant, tests only): each id makes one step take a
 * known-wrong form, so that the tests can show that the pins reject it; id
 * 0, the default, runs every step as stated above.
 *
 * Threads (OpenMP, optional): loops over independent rows or blocks carry a
 * parallel-for pragma and nothing else changes; every row or block is
 * computed by the same statements in the same order whatever the thread
 * count, and the reductions (norms, inner products) stay serial, so results
 * are bitwise identical for any number of threads (ora_set_threads).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>
#ifdef _OPENMP
#include <omp.h>
#endif

void ora_set_threads(int n) {
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}
int ora_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

#define ORA_MAXLEV 24

/* planted mistakes (see the header) */
enum {
    PL_NONE = 0,
    PL_PRESCALE_OFF,      /* the setup without W (Sec. 2.3.1) */
    PL_UPDATE_SIGN,       /* E_b + Lambda R_b instead of E_b - Lambda R_b (Alg. 2) */
    PL_LAMBDA_T,          /* every block stores Lambda_b^T */
    PL_SMOOTH_T,          /* the forward application takes Lambda^T */
    PL_COLOUR_ORDER,      /* the forward application runs its colours backwards */
    PL_REVERSE_ORDER,     /* the reverse application keeps the forward step order */
    PL_SMOOTH_SIGN,       /* the smoother adds Lambda (A x - b) */
    PL_INTERP_ONE_SIDED,  /* an even fine node interpolates from one coarse node */
    PL_RESTRICT_UNSCALED, /* R = P^T beside a Galerkin product scaled 2^{-d} */
    PL_COARSE_CHOL,       /* the coarsest solve takes Cholesky of a nonsymmetric A_c */
    PL_TRUNC_SMALLEST,    /* truncation keeps the alpha smallest column blocks */
    PL_MINNORM_OFF,       /* the block least squares without the minimum-norm cutoff */
    PL_OVERLAP_SUM,       /* overlapping rows summed instead of averaged over theta */
    PL_STOKES_Q2,         /* the L^2 pressure weight sums |a| w without squaring */
    PL_SPD_NO_UPPER,      /* the SPD projection clips at 0 only, not at D^{-1} */
    PL_PCG_BETA,          /* PCG with beta = rz_k / rz_{k+1} */
    PL_GREEDY_ASCENDING,  /* the greedy colouring visits blocks in ascending priority */
    PL_SKETCH_STALE,      /* the sketched setup never advances E S */
    PL_PRESCALE_POWER,    /* the elliptic weight 1 / A_ii instead of A_ii^{-1/2} */
    PL_OVERLAP_SMOOTH_SUM,/* the overlapping smoother sums its block corrections */
    PL_GALERKIN_RSCALE,   /* a user hierarchy's coarse operator without rscale */
    PL_PARITY,            /* red-black parity from the x block index alone */
    PL_GIVENS_SIGN,       /* left GMRES rotates H with the sign of s flipped */
    PL_RIGHT_UPDATE_V,    /* right GMRES updates x from V y instead of Z y */
    PL_INPLACE_COLOUR,    /* a setup step's blocks see the rows updated before them (serial) */
    PL_SKETCH_FIRST_T,    /* the sketch's exact first step takes C = A~_bb instead of A~_bb^T */
    PL_BOUNDARY_WRAP,     /* a Dirichlet grid wraps its stencil like a periodic one */
    PL_PROLONG_SIGN,      /* the V-cycle adds P x_c with the wrong sign */
    PL_RF_FORWARD,        /* the RF cycle pre-smooths with the forward application */
    PL_STOKES_VEL_L1,     /* the velocity weight ||a_i||_1 / a_ii instead of its square root */
    PL_SKETCH_Z_ONCE,     /* the multiplicative sketch forms A~ Y once per step, not per colour */
    PL_SPD_UNWEIGHTED,    /* the SPD projection takes D = I instead of A~_bb */
};
static int planted = PL_NONE;
void ora_plant(int id) { planted = id; }

/* ------------------------------------------------------------------ CSR */
typedef struct {
    int n, m;
    int64_t *rp;
    int *ci;
    double *v;
} csr;

static void *xmalloc(size_t sz) {
    void *p = malloc(sz ? sz : 1);
    if (!p) { fprintf(stderr, "oracle: out of memory (%zu bytes)\n", sz); abort(); }
    return p;
}
static void *xcalloc(size_t n, size_t sz) {
    void *p = calloc(n ? n : 1, sz ? sz : 1);
    if (!p) { fprintf(stderr, "oracle: out of memory\n"); abort(); }
    return p;
}
static void csr_free(csr *a) {
    free(a->rp); free(a->ci); free(a->v);
    memset(a, 0, sizeof(*a));
}

static int cmp_int(const void *a, const void *b) {
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

/* y = A x */
static void csr_matvec(const csr *A, const double *x, double *y) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < A->n; ++i) {
        double s = 0.0;
        for (int64_t p = A->rp[i]; p < A->rp[i + 1]; ++p) s += A->v[p] * x[A->ci[p]];
        y[i] = s;
    }
}

static void csr_transpose(const csr *A, csr *T) {
    T->n = A->m; T->m = A->n;
    int64_t nnz = A->rp[A->n];
    T->rp = xcalloc((size_t)T->n + 1, sizeof(int64_t));
    T->ci = xmalloc(sizeof(int) * (size_t)nnz);
    T->v = xmalloc(sizeof(double) * (size_t)nnz);
    for (int64_t p = 0; p < nnz; ++p) T->rp[A->ci[p] + 1]++;
    for (int j = 0; j < T->n; ++j) T->rp[j + 1] += T->rp[j];
    int64_t *fill = xmalloc(sizeof(int64_t) * (size_t)T->n);
    for (int j = 0; j < T->n; ++j) fill[j] = T->rp[j];
    for (int i = 0; i < A->n; ++i)
        for (int64_t p = A->rp[i]; p < A->rp[i + 1]; ++p) {
            int64_t q = fill[A->ci[p]]++;
            T->ci[q] = i; T->v[q] = A->v[p];
        }
    free(fill);
}

/* C = s * A B (Gustavson; columns sorted in each row).  Two passes over the
 * rows (count, then fill) so that rows can be formed in parallel; each row's
 * sums are accumulated in the same order either way. */
static void csr_spgemm(const csr *A, const csr *B, double s, csr *C) {
    C->n = A->n; C->m = B->m;
    C->rp = xmalloc(sizeof(int64_t) * ((size_t)A->n + 1));
    int *cnt = xmalloc(sizeof(int) * ((size_t)A->n + 1));
#pragma omp parallel
    {
        int *mark = xmalloc(sizeof(int) * (size_t)B->m);
        for (int j = 0; j < B->m; ++j) mark[j] = -1;
#pragma omp for schedule(static)
        for (int i = 0; i < A->n; ++i) {
            int c = 0;
            for (int64_t p = A->rp[i]; p < A->rp[i + 1]; ++p) {
                int k = A->ci[p];
                for (int64_t q = B->rp[k]; q < B->rp[k + 1]; ++q)
                    if (mark[B->ci[q]] != i) { mark[B->ci[q]] = i; ++c; }
            }
            cnt[i] = c;
        }
        free(mark);
    }
    C->rp[0] = 0;
    for (int i = 0; i < A->n; ++i) C->rp[i + 1] = C->rp[i] + cnt[i];
    int64_t nnz = C->rp[A->n];
    C->ci = xmalloc(sizeof(int) * (size_t)(nnz ? nnz : 1));
    C->v = xmalloc(sizeof(double) * (size_t)(nnz ? nnz : 1));
#pragma omp parallel
    {
        int *mark = xmalloc(sizeof(int) * (size_t)B->m);
        double *acc = xcalloc((size_t)B->m, sizeof(double));
        int *list = xmalloc(sizeof(int) * (size_t)B->m);
        for (int j = 0; j < B->m; ++j) mark[j] = -1;
#pragma omp for schedule(static)
        for (int i = 0; i < A->n; ++i) {
            int c = 0;
            for (int64_t p = A->rp[i]; p < A->rp[i + 1]; ++p) {
                int k = A->ci[p];
                double a = A->v[p];
                for (int64_t q = B->rp[k]; q < B->rp[k + 1]; ++q) {
                    int j = B->ci[q];
                    if (mark[j] != i) { mark[j] = i; list[c++] = j; acc[j] = 0.0; }
                    acc[j] += a * B->v[q];
                }
            }
            qsort(list, (size_t)c, sizeof(int), cmp_int);
            int64_t o = C->rp[i];
            for (int t = 0; t < c; ++t) { C->ci[o + t] = list[t]; C->v[o + t] = s * acc[list[t]]; }
        }
        free(mark); free(acc); free(list);
    }
    free(cnt);
}

/* Structured stencil -> CSR.  Row i = ix + nx*(iy + ny*iz); entry s couples
 * i to i + off[s].  Dirichlet: neighbours outside the interior grid are
 * eliminated (dropped).  Periodic: indices wrap; duplicate columns (tiny
 * grids) are summed. */
static void csr_from_stencil(const int n3[3], int nst, const int *off, const double *coeff,
                             int periodic, csr *A) {
    int nx = n3[0], ny = n3[1], nz = n3[2];
    int N = nx * ny * nz;
    A->n = A->m = N;
    A->rp = xmalloc(sizeof(int64_t) * ((size_t)N + 1));
    A->ci = xmalloc(sizeof(int) * (size_t)N * (size_t)nst);
    A->v = xmalloc(sizeof(double) * (size_t)N * (size_t)nst);
    int64_t nnz = 0;
    A->rp[0] = 0;
    int *cols = xmalloc(sizeof(int) * (size_t)nst);
    double *vals = xmalloc(sizeof(double) * (size_t)nst);
    for (int iz = 0; iz < nz; ++iz)
        for (int iy = 0; iy < ny; ++iy)
            for (int ix = 0; ix < nx; ++ix) {
                int i = ix + nx * (iy + ny * iz);
                int cnt = 0;
                for (int s = 0; s < nst; ++s) {
                    int jx = ix + off[3 * s], jy = iy + off[3 * s + 1], jz = iz + off[3 * s + 2];
                    if (periodic || planted == PL_BOUNDARY_WRAP) {
                        jx = (jx % nx + nx) % nx; jy = (jy % ny + ny) % ny; jz = (jz % nz + nz) % nz;
                    } else if (jx < 0 || jx >= nx || jy < 0 || jy >= ny || jz < 0 || jz >= nz) {
                        continue;
                    }
                    int j = jx + nx * (jy + ny * jz);
                    double a = coeff[(size_t)s * N + i];
                    int found = -1;
                    for (int t = 0; t < cnt; ++t) if (cols[t] == j) found = t;
                    if (found >= 0) vals[found] += a;
                    else { cols[cnt] = j; vals[cnt] = a; ++cnt; }
                }
                /* insertion sort by column */
                for (int a = 1; a < cnt; ++a) {
                    int c = cols[a]; double v = vals[a]; int b = a - 1;
                    while (b >= 0 && cols[b] > c) { cols[b + 1] = cols[b]; vals[b + 1] = vals[b]; --b; }
                    cols[b + 1] = c; vals[b + 1] = v;
                }
                for (int t = 0; t < cnt; ++t) { A->ci[nnz] = cols[t]; A->v[nnz] = vals[t]; ++nnz; }
                A->rp[i + 1] = nnz;
            }
    free(cols); free(vals);
}

/* 1D node-centred interpolation on interior nodes (SM Sec. 4.1, bilinear /
 * trilinear in tensor form).  Coarse interior nodes are the fine nodes with
 * even 1-based index: coarse c (0-based) sits on fine 2c+1 (0-based).  A fine
 * node with odd 1-based index takes half of each coarse neighbour; the
 * Dirichlet boundary contributes zero. */
static int p1d_entries(int f, int nc, int *c, double *w) {
    if (f % 2 == 1) { c[0] = (f - 1) / 2; w[0] = 1.0; return 1; }
    int k = 0;
    int lo = f / 2 - 1, hi = f / 2;
    if (lo >= 0 && lo < nc && planted != PL_INTERP_ONE_SIDED) { c[k] = lo; w[k] = 0.5; ++k; }
    if (hi >= 0 && hi < nc) { c[k] = hi; w[k] = 0.5; ++k; }
    return k;
}

static void prolongation(const int nf[3], const int nc[3], int dim, csr *P) {
    int Nf = nf[0] * nf[1] * nf[2], Nc = nc[0] * nc[1] * nc[2];
    P->n = Nf; P->m = Nc;
    P->rp = xmalloc(sizeof(int64_t) * ((size_t)Nf + 1));
    P->ci = xmalloc(sizeof(int) * (size_t)Nf * 8);
    P->v = xmalloc(sizeof(double) * (size_t)Nf * 8);
    int64_t nnz = 0;
    P->rp[0] = 0;
    for (int fz = 0; fz < nf[2]; ++fz)
        for (int fy = 0; fy < nf[1]; ++fy)
            for (int fx = 0; fx < nf[0]; ++fx) {
                int cx[2], cy[2], cz[2];
                double wx[2], wy[2], wz[2];
                int kx = p1d_entries(fx, nc[0], cx, wx);
                int ky = p1d_entries(fy, nc[1], cy, wy);
                int kz;
                if (dim == 3) kz = p1d_entries(fz, nc[2], cz, wz);
                else { kz = 1; cz[0] = 0; wz[0] = 1.0; }
                int cols[8]; double vals[8]; int cnt = 0;
                for (int c = 0; c < kz; ++c)
                    for (int b = 0; b < ky; ++b)
                        for (int a = 0; a < kx; ++a) {
                            cols[cnt] = cx[a] + nc[0] * (cy[b] + nc[1] * cz[c]);
                            vals[cnt] = wx[a] * wy[b] * wz[c];
                            ++cnt;
                        }
                for (int a = 1; a < cnt; ++a) {
                    int c = cols[a]; double v = vals[a]; int b = a - 1;
                    while (b >= 0 && cols[b] > c) { cols[b + 1] = cols[b]; vals[b + 1] = vals[b]; --b; }
                    cols[b + 1] = c; vals[b + 1] = v;
                }
                for (int t = 0; t < cnt; ++t) { P->ci[nnz] = cols[t]; P->v[nnz] = vals[t]; ++nnz; }
                P->rp[fx + nf[0] * (fy + nf[1] * fz) + 1] = nnz;
            }
}

/* ---------------------------------------------------------- dense LA */
/* In-place Cholesky of the n x n row-major SPD matrix a (lower factor).
 * Returns 0, or 1 if a pivot is <= tol. */
static int chol(double *a, int n, double tol) {
    for (int j = 0; j < n; ++j) {
        double d = a[j * n + j];
        for (int k = 0; k < j; ++k) d -= a[j * n + k] * a[j * n + k];
        if (!(d > tol)) return 1;
        d = sqrt(d);
        a[j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double s = a[i * n + j];
            for (int k = 0; k < j; ++k) s -= a[i * n + k] * a[j * n + k];
            a[i * n + j] = s / d;
        }
    }
    return 0;
}
/* Solve L L^T y = r in place (L from chol). */
static void chol_solve(const double *L, int n, double *y) {
    for (int i = 0; i < n; ++i) {
        double s = y[i];
        for (int k = 0; k < i; ++k) s -= L[i * n + k] * y[k];
        y[i] = s / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * y[k];
        y[i] = s / L[i * n + i];
    }
}
/* LU with partial pivoting in place; returns 0 or 1 if singular. */
static int lu(double *a, int n, int *piv) {
    for (int k = 0; k < n; ++k) {
        int p = k; double best = fabs(a[k * n + k]);
        for (int i = k + 1; i < n; ++i) if (fabs(a[i * n + k]) > best) { best = fabs(a[i * n + k]); p = i; }
        piv[k] = p;
        if (best == 0.0) return 1;
        if (p != k) for (int j = 0; j < n; ++j) { double t = a[k * n + j]; a[k * n + j] = a[p * n + j]; a[p * n + j] = t; }
        for (int i = k + 1; i < n; ++i) {
            double f = a[i * n + k] / a[k * n + k];
            a[i * n + k] = f;
            for (int j = k + 1; j < n; ++j) a[i * n + j] -= f * a[k * n + j];
        }
    }
    return 0;
}
static void lu_solve(const double *a, int n, const int *piv, double *y) {
    for (int k = 0; k < n; ++k) if (piv[k] != k) { double t = y[k]; y[k] = y[piv[k]]; y[piv[k]] = t; }
    for (int i = 0; i < n; ++i) { double s = y[i]; for (int k = 0; k < i; ++k) s -= a[i * n + k] * y[k]; y[i] = s; }
    for (int i = n - 1; i >= 0; --i) { double s = y[i]; for (int k = i + 1; k < n; ++k) s -= a[i * n + k] * y[k]; y[i] = s / a[i * n + i]; }
}
/* Cyclic Jacobi eigendecomposition of a symmetric n x n matrix a (destroyed):
 * eigenvalues in ev, eigenvectors in the columns of q. */
static void sym_eig(double *a, int n, double *ev, double *q) {
    for (int i = 0; i < n * n; ++i) q[i] = 0.0;
    for (int i = 0; i < n; ++i) q[i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < n; ++i) for (int j = i + 1; j < n; ++j) off += a[i * n + j] * a[i * n + j];
        if (off < 1e-300) break;
        for (int p = 0; p < n; ++p)
            for (int r = p + 1; r < n; ++r) {
                double apr = a[p * n + r];
                if (apr == 0.0) continue;
                double theta = (a[r * n + r] - a[p * n + p]) / (2.0 * apr);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {
                    double akp = a[k * n + p], akr = a[k * n + r];
                    a[k * n + p] = c * akp - s * akr;
                    a[k * n + r] = s * akp + c * akr;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = a[p * n + k], ark = a[r * n + k];
                    a[p * n + k] = c * apk - s * ark;
                    a[r * n + k] = s * apk + c * ark;
                }
                for (int k = 0; k < n; ++k) {
                    double qkp = q[k * n + p], qkr = q[k * n + r];
                    q[k * n + p] = c * qkp - s * qkr;
                    q[k * n + r] = s * qkp + c * qkr;
                }
            }
    }
    for (int i = 0; i < n; ++i) ev[i] = a[i * n + i];
}

/* Lam (n x n) = C G^{-1} for SPD-or-semidefinite G: normal equations with
 * Cholesky; if a pivot falls to <= 1e-14 tr(G), the minimum-norm solution
 * C G^+ from the symmetric eigendecomposition. */
static void ls_solve_block(const double *G, const double *C, int n, double *Lam) {
    double tr = 0.0;
    for (int i = 0; i < n; ++i) tr += G[i * n + i];
    double tol = planted == PL_MINNORM_OFF ? 0.0 : 1e-14 * tr;
    double *L = xmalloc(sizeof(double) * (size_t)n * n);
    memcpy(L, G, sizeof(double) * (size_t)n * n);
    double *y = xmalloc(sizeof(double) * (size_t)n);
    if (tr > 0.0 && chol(L, n, tol) == 0) {
        for (int p = 0; p < n; ++p) {
            for (int q = 0; q < n; ++q) y[q] = C[p * n + q];
            chol_solve(L, n, y);
            for (int q = 0; q < n; ++q) Lam[p * n + q] = y[q];
        }
    } else {
        double *ev = xmalloc(sizeof(double) * (size_t)n), *Q = xmalloc(sizeof(double) * (size_t)n * n);
        memcpy(L, G, sizeof(double) * (size_t)n * n);
        sym_eig(L, n, ev, Q);
        /* G^+ = Q diag(1/ev, ev > tol) Q^T */
        for (int p = 0; p < n; ++p)
            for (int q = 0; q < n; ++q) {
                double s = 0.0;
                for (int k = 0; k < n; ++k) {
                    if (!(ev[k] > tol)) continue;
                    double cq = 0.0; /* (C Q)_{p,k} */
                    for (int m = 0; m < n; ++m) cq += C[p * n + m] * Q[m * n + k];
                    s += cq * Q[q * n + k] / ev[k];
                }
                Lam[p * n + q] = s;
            }
        free(ev); free(Q);
    }
    free(L); free(y);
}

/* The SPD projection of a block of Lambda~ for PCG (SM "On preconditioned
 * conjugate gradient": Lambda symmetric, I - Lambda A a contraction, the
 * projection guided by block Jacobi), read as: the nearest matrix, in the
 * Frobenius norm weighted by D = A~_bb (the block's diagonal block of the
 * prescaled operator), to the symmetric part of L among the matrices
 * 0 <= X <= D^{-1}, i.e. between zero and the block-Jacobi block.  With
 * D = U diag(d) U^T, M = D^{1/2} sym(L) D^{1/2} = Q diag(m) Q^T, the result
 * is D^{-1/2} Q diag(clip(m, 0, 1)) Q^T D^{-1/2}.  When D is not positive
 * definite the Frobenius-nearest positive semidefinite matrix is taken
 * (the symmetric part with its negative eigenvalues set to zero; Higham
 * 1988). */
static void project_spd_block(double *L, const double *D, int n) {
    double *S = xmalloc(sizeof(double) * (size_t)n * n), *Q = xmalloc(sizeof(double) * (size_t)n * n);
    double *U = xmalloc(sizeof(double) * (size_t)n * n), *T = xmalloc(sizeof(double) * (size_t)n * n);
    double *ev = xmalloc(sizeof(double) * (size_t)n), *dv = xmalloc(sizeof(double) * (size_t)n);
    double *Dh = xmalloc(sizeof(double) * (size_t)n * n), *Di = xmalloc(sizeof(double) * (size_t)n * n);
    for (int p = 0; p < n; ++p)
        for (int q = 0; q < n; ++q) S[p * n + q] = 0.5 * (L[p * n + q] + L[q * n + p]);
    memcpy(T, D, sizeof(double) * (size_t)n * n);
    sym_eig(T, n, dv, U);
    int pd = 1;
    for (int k = 0; k < n; ++k) if (!(dv[k] > 0.0)) pd = 0;
    if (pd) {
        for (int p = 0; p < n; ++p)
            for (int q = 0; q < n; ++q) {
                double a = 0.0, b = 0.0;
                for (int k = 0; k < n; ++k) {
                    a += U[p * n + k] * sqrt(dv[k]) * U[q * n + k];
                    b += U[p * n + k] / sqrt(dv[k]) * U[q * n + k];
                }
                Dh[p * n + q] = a;
                Di[p * n + q] = b;
            }
        /* T = Dh S Dh */
        for (int p = 0; p < n; ++p)
            for (int q = 0; q < n; ++q) {
                double a = 0.0;
                for (int r = 0; r < n; ++r)
                    for (int t = 0; t < n; ++t) a += Dh[p * n + r] * S[r * n + t] * Dh[t * n + q];
                T[p * n + q] = a;
            }
        sym_eig(T, n, ev, Q);
        for (int k = 0; k < n; ++k)
            ev[k] = ev[k] < 0.0 ? 0.0 : (ev[k] > 1.0 && planted != PL_SPD_NO_UPPER ? 1.0 : ev[k]);
        /* S = Q diag(ev) Q^T, then L = Di S Di */
        for (int p = 0; p < n; ++p)
            for (int q = 0; q < n; ++q) {
                double a = 0.0;
                for (int k = 0; k < n; ++k) a += Q[p * n + k] * ev[k] * Q[q * n + k];
                S[p * n + q] = a;
            }
        for (int p = 0; p < n; ++p)
            for (int q = 0; q < n; ++q) {
                double a = 0.0;
                for (int r = 0; r < n; ++r)
                    for (int t = 0; t < n; ++t) a += Di[p * n + r] * S[r * n + t] * Di[t * n + q];
                L[p * n + q] = a;
            }
    } else {
        memcpy(T, S, sizeof(double) * (size_t)n * n);
        sym_eig(T, n, ev, Q);
        for (int p = 0; p < n; ++p)
            for (int q = 0; q < n; ++q) {
                double a = 0.0;
                for (int k = 0; k < n; ++k)
                    if (ev[k] > 0.0) a += Q[p * n + k] * ev[k] * Q[q * n + k];
                L[p * n + q] = a;
            }
    }
    free(S); free(Q); free(U); free(T); free(ev); free(dv); free(Dh); free(Di);
}

/* ----------------------------------------------------- hierarchy */
typedef struct {
    int dim, nlev, periodic, bs;
    int n3[ORA_MAXLEV][3];
    csr A[ORA_MAXLEV];
    csr P[ORA_MAXLEV];  /* P[l]: level l+1 -> level l */
    csr R[ORA_MAXLEV];  /* rscale * P[l]^T */
    double rscale;
    /* block partition per level */
    int nb[ORA_MAXLEV];
    int *bptr[ORA_MAXLEV], *bidx[ORA_MAXLEV], *bpar[ORA_MAXLEV];
    int ncol[ORA_MAXLEV];  /* colours of the multiplicative cascade per level (red-black: 2) */
    int *field[ORA_MAXLEV];  /* per unknown: 0 velocity / scalar, 1 pressure (constraint); NULL: all 0 */
    int overlap[ORA_MAXLEV]; /* the blocks overlap (a node in several blocks) */
    /* coarsest-level dense factor */
    int cn, cspd;
    double *cfac;
    int *cpiv;
} ora_hier;

/* Blocks of bs^d nodes (partial at the upper edges); block (bx,by,bz) has
 * red-black parity (bx+1)+(by+1)[+(bz+1)] mod 2 (colour 0 = even). */
static void make_blocks(ora_hier *h, int l) {
    int nx = h->n3[l][0], ny = h->n3[l][1], nz = h->n3[l][2], bs = h->bs;
    int nbx = (nx + bs - 1) / bs, nby = (ny + bs - 1) / bs;
    int nbz = h->dim == 3 ? (nz + bs - 1) / bs : 1;
    int nb = nbx * nby * nbz, N = nx * ny * nz;
    h->nb[l] = nb;
    h->bptr[l] = xcalloc((size_t)nb + 1, sizeof(int));
    h->bidx[l] = xmalloc(sizeof(int) * (size_t)N);
    h->bpar[l] = xmalloc(sizeof(int) * (size_t)nb);
    int *blk = xmalloc(sizeof(int) * (size_t)N);
    for (int iz = 0; iz < nz; ++iz)
        for (int iy = 0; iy < ny; ++iy)
            for (int ix = 0; ix < nx; ++ix) {
                int bz = h->dim == 3 ? iz / bs : 0;
                int b = ix / bs + nbx * (iy / bs + nby * bz);
                blk[ix + nx * (iy + ny * iz)] = b;
                h->bptr[l][b + 1]++;
            }
    for (int b = 0; b < nb; ++b) h->bptr[l][b + 1] += h->bptr[l][b];
    int *fill = xmalloc(sizeof(int) * (size_t)nb);
    for (int b = 0; b < nb; ++b) fill[b] = h->bptr[l][b];
    for (int i = 0; i < N; ++i) h->bidx[l][fill[blk[i]]++] = i; /* ascending i */
    for (int bz = 0; bz < nbz; ++bz)
        for (int by = 0; by < nby; ++by)
            for (int bx = 0; bx < nbx; ++bx) {
                int s = planted == PL_PARITY ? bx : (bx + 1) + (by + 1) + (h->dim == 3 ? bz + 1 : 0);
                h->bpar[l][bx + nbx * (by + nby * bz)] = s & 1;
            }
    free(fill); free(blk);
}

static void factor_coarsest(ora_hier *h) {
    int l = h->nlev - 1;
    const csr *A = &h->A[l];
    int n = A->n;
    h->cn = n;
    h->cfac = xcalloc((size_t)n * n, sizeof(double));
    h->cpiv = xmalloc(sizeof(int) * (size_t)n);
    for (int i = 0; i < n; ++i)
        for (int64_t p = A->rp[i]; p < A->rp[i + 1]; ++p) h->cfac[(size_t)i * n + A->ci[p]] += A->v[p];
    /* Algorithm 1's bottom-level direct solve must solve A_c itself.  chol()
     * reads only the lower triangle, so it is taken only when A_c is
     * symmetric (to 1e-14 of its largest entry) and every pivot is positive;
     * otherwise LU with partial pivoting. */
    double amax = 0.0, asym = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double a = fabs(h->cfac[(size_t)i * n + j]);
            double d = fabs(h->cfac[(size_t)i * n + j] - h->cfac[(size_t)j * n + i]);
            if (a > amax) amax = a;
            if (d > asym) asym = d;
        }
    double *tmp = xmalloc(sizeof(double) * (size_t)n * n);
    memcpy(tmp, h->cfac, sizeof(double) * (size_t)n * n);
    if ((asym <= 1e-14 * amax || planted == PL_COARSE_CHOL) && chol(tmp, n, 0.0) == 0) {
        h->cspd = 1;
        memcpy(h->cfac, tmp, sizeof(double) * (size_t)n * n);
    } else {
        h->cspd = 0;
        lu(h->cfac, n, h->cpiv);
    }
    free(tmp);
}

/* coarsen_mode: 0 -> R = 2^{-d} P^T (SM Sec. 4.1); 1 -> R = P^T (Alg. 1 as
 * printed).  The V-cycle is invariant to this scale (tests pin that). */
ora_hier *ora_hier_create(int dim, const int *n3, int nst, const int *off, const double *coeff,
                          int periodic, int bs, int coarse_max, int max_levels, int rscale_mode) {
    ora_hier *h = xcalloc(1, sizeof(ora_hier));
    h->dim = dim; h->periodic = periodic; h->bs = bs < 1 ? 1 : bs;
    h->rscale = rscale_mode == 1 ? 1.0 : 1.0 / (double)(1 << dim);
    h->n3[0][0] = n3[0]; h->n3[0][1] = n3[1]; h->n3[0][2] = dim == 3 ? n3[2] : 1;
    csr_from_stencil(h->n3[0], nst, off, coeff, periodic, &h->A[0]);
    int l = 0;
    if (max_levels < 1) max_levels = ORA_MAXLEV;
    if (max_levels > ORA_MAXLEV) max_levels = ORA_MAXLEV;
    while (!periodic && l + 1 < max_levels) {
        int mx = h->n3[l][0], mn = h->n3[l][0];
        for (int d = 1; d < dim; ++d) {
            if (h->n3[l][d] > mx) mx = h->n3[l][d];
            if (h->n3[l][d] < mn) mn = h->n3[l][d];
        }
        if (mx <= coarse_max || mn < 2) break;
        int nc[3] = {h->n3[l][0] / 2, h->n3[l][1] / 2, dim == 3 ? h->n3[l][2] / 2 : 1};
        prolongation(h->n3[l], nc, dim, &h->P[l]);
        csr Pt, AP;
        csr_transpose(&h->P[l], &Pt);
        csr_spgemm(&h->A[l], &h->P[l], 1.0, &AP);
        csr_spgemm(&Pt, &AP, h->rscale, &h->A[l + 1]);
        csr_transpose(&h->P[l], &h->R[l]);
        if (planted != PL_RESTRICT_UNSCALED)
            for (int64_t p = 0; p < h->R[l].rp[h->R[l].n]; ++p) h->R[l].v[p] *= h->rscale;
        csr_free(&Pt); csr_free(&AP);
        ++l;
        h->n3[l][0] = nc[0]; h->n3[l][1] = nc[1]; h->n3[l][2] = nc[2];
    }
    h->nlev = l + 1;
    for (int k = 0; k < h->nlev; ++k) { make_blocks(h, k); h->ncol[k] = 2; }
    factor_coarsest(h);
    return h;
}

void ora_hier_free(ora_hier *h) {
    if (!h) return;
    for (int l = 0; l < h->nlev; ++l) {
        csr_free(&h->A[l]); csr_free(&h->P[l]); csr_free(&h->R[l]);
        free(h->bptr[l]); free(h->bidx[l]); free(h->bpar[l]); free(h->field[l]);
    }
    free(h->cfac); free(h->cpiv); free(h);
}
int ora_hier_nlev(const ora_hier *h) { return h->nlev; }
void ora_hier_dims(const ora_hier *h, int l, int *n3) { for (int d = 0; d < 3; ++d) n3[d] = h->n3[l][d]; }
int64_t ora_hier_nnz(const ora_hier *h, int l) { return h->A[l].rp[h->A[l].n]; }
void ora_hier_csr(const ora_hier *h, int l, int64_t *rp, int *ci, double *v) {
    const csr *A = &h->A[l];
    memcpy(rp, A->rp, sizeof(int64_t) * ((size_t)A->n + 1));
    memcpy(ci, A->ci, sizeof(int) * (size_t)A->rp[A->n]);
    memcpy(v, A->v, sizeof(double) * (size_t)A->rp[A->n]);
}
int ora_hier_nblocks(const ora_hier *h, int l) { return h->nb[l]; }
int ora_hier_nbidx(const ora_hier *h, int l) { return h->bptr[l][h->nb[l]]; }
void ora_hier_blocks(const ora_hier *h, int l, int *bptr, int *bidx, int *bpar) {
    memcpy(bptr, h->bptr[l], sizeof(int) * ((size_t)h->nb[l] + 1));
    memcpy(bidx, h->bidx[l], sizeof(int) * (size_t)h->bptr[l][h->nb[l]]);
    memcpy(bpar, h->bpar[l], sizeof(int) * (size_t)h->nb[l]);
}

/* ----------------------------------------- hierarchy from a CSR operator
 * The block partition of A x = b is the user's (Sec. 2), and so are the
 * hierarchy's transfers (Sec. 2.4): the user gives the finest operator and
 * one interpolation P_l (N_l x N_{l+1}) per coarser level; the coarse
 * operators are Galerkin, A_{l+1} = R_l A_l P_l with R_l = rscale P_l^T.
 * Blocks: the user's partition of level 0, point blocks on coarser levels.
 * The multiplicative cascade uses a greedy colouring of each level's block
 * graph (blocks adjacent when A couples them in either direction): blocks
 * in decreasing order of a pseudo-random priority (ties: smaller index
 * first) take the smallest colour that no adjacent, already coloured block
 * holds -- the colouring a parallel Jones-Plassmann pass with the same
 * priorities produces.  Block b of level l has priority mix(seed + (c + 1) g)
 * (SplitMix64, counter c = l 2^40 + b). */
static uint64_t sm64_mix(uint64_t z);
static uint64_t block_prio(uint64_t seed, int l, int b) {
    uint64_t c = ((uint64_t)l << 40) + (uint64_t)b;
    return sm64_mix(seed + (c + 1) * 0x9E3779B97F4A7C15ULL);
}
uint64_t ora_block_prio(uint64_t seed, int l, int b) { return block_prio(seed, l, b); }

static void csr_copy_in(csr *A, int n, int m, const int64_t *rp, const int *ci, const double *v) {
    A->n = n; A->m = m;
    int64_t nnz = rp[n];
    A->rp = xmalloc(sizeof(int64_t) * ((size_t)n + 1));
    A->ci = xmalloc(sizeof(int) * (size_t)(nnz ? nnz : 1));
    A->v = xmalloc(sizeof(double) * (size_t)(nnz ? nnz : 1));
    memcpy(A->rp, rp, sizeof(int64_t) * ((size_t)n + 1));
    memcpy(A->ci, ci, sizeof(int) * (size_t)nnz);
    memcpy(A->v, v, sizeof(double) * (size_t)nnz);
}

ora_hier *ora_ghier_new(int N, const int64_t *rp, const int *ci, const double *v, double rscale) {
    ora_hier *h = xcalloc(1, sizeof(ora_hier));
    h->dim = 0; h->bs = 0; h->rscale = rscale; h->nlev = 1;
    h->n3[0][0] = N; h->n3[0][1] = 1; h->n3[0][2] = 1;
    csr_copy_in(&h->A[0], N, N, rp, ci, v);
    return h;
}

/* Appends level l+1 below the current coarsest level l: P is N_l x Nc. */
int ora_ghier_add_level(ora_hier *h, int Nc, const int64_t *prp, const int *pci, const double *pv) {
    int l = h->nlev - 1;
    if (h->nlev >= ORA_MAXLEV) return -1;
    csr_copy_in(&h->P[l], h->A[l].n, Nc, prp, pci, pv);
    csr Pt, AP;
    csr_transpose(&h->P[l], &Pt);
    csr_spgemm(&h->A[l], &h->P[l], 1.0, &AP);
    csr_spgemm(&Pt, &AP, planted == PL_GALERKIN_RSCALE ? 1.0 : h->rscale, &h->A[l + 1]);
    csr_transpose(&h->P[l], &h->R[l]);
    for (int64_t p = 0; p < h->R[l].rp[h->R[l].n]; ++p) h->R[l].v[p] *= h->rscale;
    csr_free(&Pt); csr_free(&AP);
    h->nlev = l + 2;
    h->n3[l + 1][0] = Nc; h->n3[l + 1][1] = 1; h->n3[l + 1][2] = 1;
    return 0;
}

/* The user's block partition of level 0 (every node in exactly one block;
 * the nodes of a block are used in the order given).  Returns -1 if it is
 * not a partition. */
int ora_ghier_set_blocks(ora_hier *h, int l, int nb, const int *bptr, const int *bidx) {
    if (l < 0 || l >= h->nlev) return -1;
    int N = h->A[l].n;
    if (nb < 1 || bptr[0] != 0) return -1;
    for (int b = 0; b < nb; ++b) if (bptr[b + 1] <= bptr[b]) return -1;
    int M = bptr[nb];
    /* every node in at least one block, no node twice in one block; a node
     * in several blocks makes the blocks overlapping (Sec. 3.6.2) */
    int *cnt = xcalloc((size_t)N, sizeof(int)), *last = xmalloc(sizeof(int) * (size_t)N);
    for (int i = 0; i < N; ++i) last[i] = -1;
    int over = 0, bad = 0;
    for (int b = 0; b < nb && !bad; ++b)
        for (int p = bptr[b]; p < bptr[b + 1]; ++p) {
            int i = bidx[p];
            if (i < 0 || i >= N || last[i] == b) { bad = 1; break; }
            last[i] = b;
            if (cnt[i]++) over = 1;
        }
    for (int i = 0; i < N && !bad; ++i) if (!cnt[i]) bad = 1;
    free(cnt); free(last);
    if (bad) return -1;
    free(h->bptr[l]); free(h->bidx[l]);
    h->nb[l] = nb;
    h->overlap[l] = over;
    h->bptr[l] = xmalloc(sizeof(int) * ((size_t)nb + 1));
    h->bidx[l] = xmalloc(sizeof(int) * (size_t)M);
    memcpy(h->bptr[l], bptr, sizeof(int) * ((size_t)nb + 1));
    memcpy(h->bidx[l], bidx, sizeof(int) * (size_t)M);
    return 0;
}
int ora_hier_overlap(const ora_hier *h, int l) { return h->overlap[l]; }

/* node -> blocks containing it, in ascending block order (CSR: nptr [N+1],
 * nblk / nloc [M]: the block and the node's position in it) */
static void node_blocks(const ora_hier *h, int l, int **nptr, int **nblk, int **nloc) {
    int N = h->A[l].n, nb = h->nb[l], M = h->bptr[l][nb];
    *nptr = xcalloc((size_t)N + 1, sizeof(int));
    *nblk = xmalloc(sizeof(int) * (size_t)M);
    *nloc = xmalloc(sizeof(int) * (size_t)M);
    for (int p = 0; p < M; ++p) (*nptr)[h->bidx[l][p] + 1]++;
    for (int i = 0; i < N; ++i) (*nptr)[i + 1] += (*nptr)[i];
    int *fill = xmalloc(sizeof(int) * (size_t)N);
    for (int i = 0; i < N; ++i) fill[i] = (*nptr)[i];
    for (int b = 0; b < nb; ++b)
        for (int p = h->bptr[l][b]; p < h->bptr[l][b + 1]; ++p) {
            int q = fill[h->bidx[l][p]]++;
            (*nblk)[q] = b;
            (*nloc)[q] = p - h->bptr[l][b];
        }
    free(fill);
}

/* Field of every finest unknown (0 velocity or scalar, 1 pressure); the
 * coarse unknowns take the field of the fine unknowns P maps them to. */
void ora_ghier_set_fields(ora_hier *h, const int *field) {
    int N = h->A[0].n;
    free(h->field[0]);
    h->field[0] = xmalloc(sizeof(int) * (size_t)N);
    memcpy(h->field[0], field, sizeof(int) * (size_t)N);
}

typedef struct { uint64_t p; int b; } prio_t;
static int cmp_prio(const void *a, const void *b) {
    const prio_t *x = a, *y = b;
    if (x->p != y->p) return (x->p > y->p) != (planted == PL_GREEDY_ASCENDING) ? -1 : 1; /* larger priority first */
    return (x->b > y->b) - (x->b < y->b);          /* then smaller index */
}

static void greedy_colour(ora_hier *h, int l, uint64_t seed) {
    const csr *A = &h->A[l];
    int nb = h->nb[l];
    int *nptr, *nblk, *nloc;
    node_blocks(h, l, &nptr, &nblk, &nloc);
    /* symmetrised block adjacency as lists (duplicates allowed): blocks b and
     * c touch when a row of b couples to a node of c, or they share a node */
    int *deg = xcalloc((size_t)nb + 1, sizeof(int));
    for (int b = 0; b < nb; ++b)
        for (int p = h->bptr[l][b]; p < h->bptr[l][b + 1]; ++p) {
            int i = h->bidx[l][p];
            for (int64_t q = A->rp[i] - 1; q < A->rp[i + 1]; ++q) {  /* q = rp[i] - 1: the node itself */
                int j = q < A->rp[i] ? i : A->ci[q];
                for (int u = nptr[j]; u < nptr[j + 1]; ++u)
                    if (nblk[u] != b) { deg[b + 1]++; deg[nblk[u] + 1]++; }
            }
        }
    for (int b = 0; b < nb; ++b) deg[b + 1] += deg[b];
    int *adj = xmalloc(sizeof(int) * (size_t)(deg[nb] ? deg[nb] : 1));
    int *fill = xmalloc(sizeof(int) * (size_t)nb);
    for (int b = 0; b < nb; ++b) fill[b] = deg[b];
    for (int b = 0; b < nb; ++b)
        for (int p = h->bptr[l][b]; p < h->bptr[l][b + 1]; ++p) {
            int i = h->bidx[l][p];
            for (int64_t q = A->rp[i] - 1; q < A->rp[i + 1]; ++q) {
                int j = q < A->rp[i] ? i : A->ci[q];
                for (int u = nptr[j]; u < nptr[j + 1]; ++u) {
                    int c = nblk[u];
                    if (c == b) continue;
                    adj[fill[b]++] = c; adj[fill[c]++] = b;
                }
            }
        }
    free(nptr); free(nblk); free(nloc);
    int *blk = NULL;
    prio_t *ord = xmalloc(sizeof(prio_t) * (size_t)nb);
    for (int b = 0; b < nb; ++b) { ord[b].p = block_prio(seed, l, b); ord[b].b = b; }
    qsort(ord, (size_t)nb, sizeof(prio_t), cmp_prio);
    int *col = h->bpar[l];
    for (int b = 0; b < nb; ++b) col[b] = -1;
    int maxc = 0;
    char used[256];
    for (int k = 0; k < nb; ++k) {
        int b = ord[k].b;
        memset(used, 0, sizeof(used));
        for (int q = deg[b]; q < deg[b + 1]; ++q)
            if (col[adj[q]] >= 0 && col[adj[q]] < 256) used[col[adj[q]]] = 1;
        int c = 0;
        while (c < 255 && used[c]) ++c;
        col[b] = c;
        if (c + 1 > maxc) maxc = c + 1;
    }
    h->ncol[l] = maxc;
    free(blk); free(deg); free(adj); free(fill); free(ord);
}

/* Point blocks on every level without a partition, the colourings, and the
 * coarsest factorisation. */
int ora_ghier_finish(ora_hier *h, uint64_t seed) {
    for (int l = 0; l + 1 < h->nlev && h->field[0]; ++l) {
        const csr *P = &h->P[l];
        int Nc = P->m;
        h->field[l + 1] = xmalloc(sizeof(int) * (size_t)Nc);
        for (int j = 0; j < Nc; ++j) h->field[l + 1][j] = -1;
        for (int i = 0; i < P->n; ++i)
            for (int64_t p = P->rp[i]; p < P->rp[i + 1]; ++p) {
                int *f = &h->field[l + 1][P->ci[p]];
                if (*f >= 0 && *f != h->field[l][i]) return -1; /* a coarse unknown of two fields */
                *f = h->field[l][i];
            }
        for (int j = 0; j < Nc; ++j) if (h->field[l + 1][j] < 0) h->field[l + 1][j] = 0;
    }
    for (int l = 0; l < h->nlev; ++l) {
        int N = h->A[l].n;
        if (!h->bptr[l]) {
            h->nb[l] = N;
            h->bptr[l] = xmalloc(sizeof(int) * ((size_t)N + 1));
            h->bidx[l] = xmalloc(sizeof(int) * (size_t)N);
            for (int i = 0; i <= N; ++i) h->bptr[l][i] = i;
            for (int i = 0; i < N; ++i) h->bidx[l][i] = i;
        }
        free(h->bpar[l]);
        h->bpar[l] = xmalloc(sizeof(int) * (size_t)h->nb[l]);
        greedy_colour(h, l, seed);
    }
    factor_coarsest(h);
    return 0;
}
int ora_hier_ncol(const ora_hier *h, int l) { return h->ncol[l]; }

/* ------------------------------------------------------- cascade setup */
typedef struct { int nnz; int *c; double *v; } srow;

typedef struct {
    int nlev;      /* levels with a smoother */
    int kind;      /* 0 additive, 1 multiplicative red-black */
    int ncol, nu;      /* ncol: the largest colour count over the levels */
    int ncl[ORA_MAXLEV]; /* colours per level (1 for the additive form) */
    int64_t lamsize[ORA_MAXLEV];
    int64_t *lamoff[ORA_MAXLEV];
    double *lam[ORA_MAXLEV];   /* [nu][lamsize]; block b row-major n_b x n_b */
    double *efrob[ORA_MAXLEV]; /* ||E~||_F after each (l,k) step, [nu*ncol+1] */
} ora_casc;

static int block_colour(const ora_hier *h, int l, int kind, int b) {
    return kind == 1 ? h->bpar[l][b] : 0;
}

/* The diagonal prescaling W of level l (Sec. 2.3; SM "Prescaling Stokes
 * problems"): mode 0 none (W = I); 1 elliptic, w_i = A_ii^{-1/2}; 2, 3, 4
 * Stokes with q = 1, 2, infinity: every velocity unknown (field 0) takes
 * w_i = sqrt(||A_{i,:}||_1) / A_ii, the 1-norm over the velocity columns of
 * its row (so that the diagonal of W A W there is ||A_{i,:}||_1 / A_ii), and
 * every pressure unknown (field 1) takes the w_k that gives its row of
 * diag(w_p) D diag(w_u) (the velocity columns) unit q-norm.  Returns -1 when
 * a weight is undefined (a non-positive diagonal or norm). */
static int prescale_weights(const ora_hier *h, int l, int mode, double *w) {
    const csr *A = &h->A[l];
    int N = A->n;
    const int *fld = h->field[l];
    for (int i = 0; i < N; ++i) {
        double d = 0.0;
        for (int64_t p = A->rp[i]; p < A->rp[i + 1]; ++p) if (A->ci[p] == i) d += A->v[p];
        if (mode == 0) w[i] = 1.0;
        else if (mode == 1) {
            if (!(d > 0.0)) return -1;
            w[i] = planted == PL_PRESCALE_POWER ? 1.0 / d : 1.0 / sqrt(d);
        } else if (!fld || fld[i] == 0) {
            double l1 = 0.0;
            for (int64_t p = A->rp[i]; p < A->rp[i + 1]; ++p)
                if (!fld || fld[A->ci[p]] == 0) l1 += fabs(A->v[p]);
            if (!(d > 0.0) || !(l1 > 0.0)) return -1;
            w[i] = planted == PL_STOKES_VEL_L1 ? l1 / d : sqrt(l1) / d;
        }
    }
    if (mode >= 2 && fld)
        for (int k = 0; k < N; ++k) {
            if (fld[k] != 1) continue;
            double nrm = 0.0;
            for (int64_t p = A->rp[k]; p < A->rp[k + 1]; ++p) {
                int j = A->ci[p];
                if (fld[j] != 0) continue;
                double a = fabs(A->v[p]) * w[j];
                if (mode == 2) nrm += a;
                else if (mode == 3) nrm += planted == PL_STOKES_Q2 ? a : a * a;
                else if (a > nrm) nrm = a;
            }
            if (mode == 3) nrm = sqrt(nrm);
            if (!(nrm > 0.0)) return -1;
            w[k] = 1.0 / nrm;
        }
    return 0;
}
int ora_prescale_weights(const ora_hier *h, int l, int mode, double *w) { return prescale_weights(h, l, mode, w); }

/* One level's cascade (Algorithm 2 / SM Algorithm).  A is the level
 * operator; lam receives nu * lamsize doubles, efrob nu*ncol+1 doubles. */
static int cascade_level(const ora_hier *h, int l, int kind, int nu, int prescale, int alpha, int spd,
                         const int64_t *lamoff, double *lam, double *efrob) {
    const csr *A0 = &h->A[l];
    int N = A0->n, nb = h->nb[l];
    const int *bptr = h->bptr[l], *bidx = h->bidx[l];
    int ncol = kind == 1 ? h->ncol[l] : 1;
    int64_t lamsize = lamoff[nb];
    /* the prescaling W (Sec. 2.3) */
    double *w = xmalloc(sizeof(double) * (size_t)N);
    if (prescale_weights(h, l, prescale, w) != 0) { free(w); return -1; }
    if (planted == PL_PRESCALE_OFF) for (int i = 0; i < N; ++i) w[i] = 1.0;
    const int over = h->overlap[l];
    if (over && alpha > 0) { free(w); return -1; }
    csr A;
    A.n = A.m = N;
    int64_t annz = A0->rp[N];
    A.rp = xmalloc(sizeof(int64_t) * ((size_t)N + 1));
    A.ci = xmalloc(sizeof(int) * (size_t)annz);
    A.v = xmalloc(sizeof(double) * (size_t)annz);
    memcpy(A.rp, A0->rp, sizeof(int64_t) * ((size_t)N + 1));
    memcpy(A.ci, A0->ci, sizeof(int) * (size_t)annz);
    for (int i = 0; i < N; ++i)
        for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p) A.v[p] = w[i] * A0->v[p] * w[A.ci[p]];
    /* overlapping additive blocks (Sec. 3.6.2): every block's new rows are
     * kept and the node rows fused by weighted averaging,
     * E_l = diag(theta)^{-1} Theta^T (Theta - Lambda Theta A) E_{l-1} */
    int *nptr = NULL, *nblk = NULL, *nloc = NULL;
    srow *bnew = NULL;
    if (over) {
        node_blocks(h, l, &nptr, &nblk, &nloc);
        bnew = xcalloc((size_t)bptr[nb], sizeof(srow));  /* per (block, row) */
    }

    /* block id of each unknown, for the truncation ranking */
    int *blk_of = xmalloc(sizeof(int) * (size_t)N);
    for (int b = 0; b < nb; ++b) for (int p = bptr[b]; p < bptr[b + 1]; ++p) blk_of[bidx[p]] = b;

    /* E_0 = I */
    srow *E = xmalloc(sizeof(srow) * (size_t)N);
    for (int i = 0; i < N; ++i) {
        E[i].nnz = 1; E[i].c = xmalloc(sizeof(int)); E[i].v = xmalloc(sizeof(double));
        E[i].c[0] = i; E[i].v[0] = 1.0;
    }
    srow *Enew = xcalloc((size_t)N, sizeof(srow));
    memset(lam, 0, sizeof(double) * (size_t)nu * (size_t)lamsize);

    double fr = 0.0;
    for (int i = 0; i < N; ++i) for (int t = 0; t < E[i].nnz; ++t) fr += E[i].v[t] * E[i].v[t];
    if (efrob) efrob[0] = sqrt(fr);

    for (int lev = 0; lev < nu; ++lev) {
        for (int k = 0; k < ncol; ++k) {
#pragma omp parallel if (planted != PL_INPLACE_COLOUR)
          {
            /* per-thread scratch: column marks and positions, block marks */
            int *mark = xmalloc(sizeof(int) * (size_t)N);
            int *pos = xmalloc(sizeof(int) * (size_t)N);
            int *bmark = xmalloc(sizeof(int) * (size_t)nb);
            int *ulist = xmalloc(sizeof(int) * (size_t)N);
            for (int i = 0; i < N; ++i) mark[i] = -1;
            for (int b = 0; b < nb; ++b) bmark[b] = -1;
            int stamp = 0;
#pragma omp for schedule(dynamic, 64)
            for (int b = 0; b < nb; ++b) {
                if (block_colour(h, l, kind, b) != k) continue;
                int nbk = bptr[b + 1] - bptr[b];
                const int *rows = bidx + bptr[b];
                /* column union U of the block rows of A E and E */
                ++stamp;
                int nu_cols = 0;
                for (int p = 0; p < nbk; ++p) {
                    int r = rows[p];
                    for (int64_t q = A.rp[r]; q < A.rp[r + 1]; ++q) {
                        const srow *Ej = &E[A.ci[q]];
                        for (int t = 0; t < Ej->nnz; ++t)
                            if (mark[Ej->c[t]] != stamp) { mark[Ej->c[t]] = stamp; ulist[nu_cols++] = Ej->c[t]; }
                    }
                    for (int t = 0; t < E[r].nnz; ++t)
                        if (mark[E[r].c[t]] != stamp) { mark[E[r].c[t]] = stamp; ulist[nu_cols++] = E[r].c[t]; }
                }
                qsort(ulist, (size_t)nu_cols, sizeof(int), cmp_int);
                for (int t = 0; t < nu_cols; ++t) pos[ulist[t]] = t;
                /* dense block rows R_b = (A E)_{b,:} and E_b */
                double *Rb = xcalloc((size_t)nbk * nu_cols, sizeof(double));
                double *Eb = xcalloc((size_t)nbk * nu_cols, sizeof(double));
                for (int p = 0; p < nbk; ++p) {
                    int r = rows[p];
                    for (int64_t q = A.rp[r]; q < A.rp[r + 1]; ++q) {
                        double a = A.v[q];
                        const srow *Ej = &E[A.ci[q]];
                        for (int t = 0; t < Ej->nnz; ++t) Rb[(size_t)p * nu_cols + pos[Ej->c[t]]] += a * Ej->v[t];
                    }
                    for (int t = 0; t < E[r].nnz; ++t) Eb[(size_t)p * nu_cols + pos[E[r].c[t]]] = E[r].v[t];
                }
                /* normal equations: Lam (R R^T) = E R^T */
                double *G = xcalloc((size_t)nbk * nbk, sizeof(double));
                double *C = xcalloc((size_t)nbk * nbk, sizeof(double));
                for (int p = 0; p < nbk; ++p)
                    for (int q = 0; q < nbk; ++q) {
                        double g = 0.0, c = 0.0;
                        for (int t = 0; t < nu_cols; ++t) {
                            g += Rb[(size_t)p * nu_cols + t] * Rb[(size_t)q * nu_cols + t];
                            c += Eb[(size_t)p * nu_cols + t] * Rb[(size_t)q * nu_cols + t];
                        }
                        G[p * nbk + q] = g; C[p * nbk + q] = c;
                    }
                double *Lb = lam + (size_t)lev * lamsize + lamoff[b];
                ls_solve_block(G, C, nbk, Lb);
                if (planted == PL_LAMBDA_T)
                    for (int p = 0; p < nbk; ++p)
                        for (int q = p + 1; q < nbk; ++q) { double t = Lb[p * nbk + q]; Lb[p * nbk + q] = Lb[q * nbk + p]; Lb[q * nbk + p] = t; }
                if (spd) {
                    double *Dbb = xcalloc((size_t)nbk * nbk, sizeof(double));
                    for (int p = 0; p < nbk; ++p)
                        for (int64_t q = A.rp[rows[p]]; q < A.rp[rows[p] + 1]; ++q)
                            for (int t = 0; t < nbk; ++t)
                                if (A.ci[q] == rows[t]) Dbb[p * nbk + t] += A.v[q];
                    if (planted == PL_SPD_UNWEIGHTED)
                        for (int p = 0; p < nbk; ++p)
                            for (int t = 0; t < nbk; ++t) Dbb[p * nbk + t] = p == t ? 1.0 : 0.0;
                    project_spd_block(Lb, Dbb, nbk);
                    free(Dbb);
                }
                /* new block rows E_b - Lam R_b */
                for (int p = 0; p < nbk; ++p)
                    for (int t = 0; t < nu_cols; ++t) {
                        double s = Eb[(size_t)p * nu_cols + t];
                        for (int q = 0; q < nbk; ++q) s -= Lb[p * nbk + q] * Rb[(size_t)q * nu_cols + t];
                        if (planted == PL_UPDATE_SIGN) s = 2.0 * Eb[(size_t)p * nu_cols + t] - s;
                        Eb[(size_t)p * nu_cols + t] = s;
                    }
                /* optional truncation: keep the alpha column blocks of largest
                 * Frobenius norm (ties: smaller block index) */
                char *keep = xmalloc((size_t)nu_cols);
                memset(keep, 1, (size_t)nu_cols);
                if (alpha > 0) {
                    int nbl = 0;
                    int *bl = xmalloc(sizeof(int) * (size_t)nu_cols);
                    double *bn = xmalloc(sizeof(double) * (size_t)nu_cols);
                    for (int t = 0; t < nu_cols; ++t) {
                        int cb = blk_of[ulist[t]];
                        if (bmark[cb] < 0) { bmark[cb] = nbl; bl[nbl] = cb; bn[nbl] = 0.0; ++nbl; }
                        for (int p = 0; p < nbk; ++p) bn[bmark[cb]] += Eb[(size_t)p * nu_cols + t] * Eb[(size_t)p * nu_cols + t];
                    }
                    if (nbl > alpha) {
                        /* selection by repeated maximum (plain, O(alpha nbl)) */
                        char *sel = xcalloc((size_t)nbl, 1);
                        for (int a = 0; a < alpha; ++a) {
                            int best = -1;
                            for (int u = 0; u < nbl; ++u) {
                                if (sel[u]) continue;
                                if (best < 0) { best = u; continue; }
                                const int larger = planted == PL_TRUNC_SMALLEST ? bn[u] < bn[best] : bn[u] > bn[best];
                                if (larger || (bn[u] == bn[best] && bl[u] < bl[best])) best = u;
                            }
                            sel[best] = 1;
                        }
                        for (int t = 0; t < nu_cols; ++t) keep[t] = sel[bmark[blk_of[ulist[t]]]];
                        free(sel);
                    }
                    for (int u = 0; u < nbl; ++u) bmark[bl[u]] = -1;
                    free(bl); free(bn);
                }
                for (int p = 0; p < nbk; ++p) {
                    int cnt = 0;
                    for (int t = 0; t < nu_cols; ++t) cnt += keep[t];
                    srow *o = (over && kind == 0) ? &bnew[bptr[b] + p] : &Enew[rows[p]];
                    o->nnz = cnt;
                    o->c = xmalloc(sizeof(int) * (size_t)(cnt ? cnt : 1));
                    o->v = xmalloc(sizeof(double) * (size_t)(cnt ? cnt : 1));
                    int u = 0;
                    for (int t = 0; t < nu_cols; ++t)
                        if (keep[t]) { o->c[u] = ulist[t]; o->v[u] = Eb[(size_t)p * nu_cols + t]; ++u; }
                    if (planted == PL_INPLACE_COLOUR && o == &Enew[rows[p]]) {
                        srow *e = &E[rows[p]];
                        free(e->c); free(e->v);
                        e->nnz = cnt;
                        e->c = xmalloc(sizeof(int) * (size_t)(cnt ? cnt : 1));
                        e->v = xmalloc(sizeof(double) * (size_t)(cnt ? cnt : 1));
                        memcpy(e->c, o->c, sizeof(int) * (size_t)cnt);
                        memcpy(e->v, o->v, sizeof(double) * (size_t)cnt);
                    }
                }
                free(keep); free(Rb); free(Eb); free(G); free(C);
            }
            free(mark); free(pos); free(bmark); free(ulist);
          }
            if (over && kind == 0) {
                /* fuse: node i's row is the average of its blocks' rows, summed in
                 * ascending block order over the union of their columns */
#pragma omp parallel
              {
                int *mk = xmalloc(sizeof(int) * (size_t)N), *ps = xmalloc(sizeof(int) * (size_t)N);
                int *ul = xmalloc(sizeof(int) * (size_t)N);
                for (int i = 0; i < N; ++i) mk[i] = -1;
#pragma omp for schedule(dynamic, 64)
                for (int i = 0; i < N; ++i) {
                    int nc = 0;
                    for (int u = nptr[i]; u < nptr[i + 1]; ++u) {
                        const srow *br = &bnew[bptr[nblk[u]] + nloc[u]];
                        for (int t = 0; t < br->nnz; ++t)
                            if (mk[br->c[t]] != i) { mk[br->c[t]] = i; ul[nc++] = br->c[t]; }
                    }
                    qsort(ul, (size_t)nc, sizeof(int), cmp_int);
                    for (int t = 0; t < nc; ++t) ps[ul[t]] = t;
                    srow *o = &Enew[i];
                    o->nnz = nc;
                    o->c = xmalloc(sizeof(int) * (size_t)(nc ? nc : 1));
                    o->v = xcalloc((size_t)(nc ? nc : 1), sizeof(double));
                    for (int t = 0; t < nc; ++t) o->c[t] = ul[t];
                    for (int u = nptr[i]; u < nptr[i + 1]; ++u) {
                        const srow *br = &bnew[bptr[nblk[u]] + nloc[u]];
                        for (int t = 0; t < br->nnz; ++t) o->v[ps[br->c[t]]] += br->v[t];
                    }
                    const double th = planted == PL_OVERLAP_SUM ? 1.0 : (double)(nptr[i + 1] - nptr[i]);
                    for (int t = 0; t < nc; ++t) o->v[t] /= th;
                }
                free(mk); free(ps); free(ul);
              }
                for (int q = 0; q < bptr[nb]; ++q) { free(bnew[q].c); free(bnew[q].v); bnew[q].c = NULL; bnew[q].v = NULL; bnew[q].nnz = 0; }
                for (int i = 0; i < N; ++i) { free(E[i].c); free(E[i].v); E[i] = Enew[i]; Enew[i].c = NULL; Enew[i].v = NULL; Enew[i].nnz = 0; }
            } else
            /* commit colour k (all blocks for the additive form) */
            for (int b = 0; b < nb; ++b) {
                if (block_colour(h, l, kind, b) != k) continue;
                for (int p = bptr[b]; p < bptr[b + 1]; ++p) {
                    int r = bidx[p];
                    free(E[r].c); free(E[r].v);
                    E[r] = Enew[r];
                    Enew[r].c = NULL; Enew[r].v = NULL; Enew[r].nnz = 0;
                }
            }
            if (efrob) {
                fr = 0.0;
                for (int i = 0; i < N; ++i) for (int t = 0; t < E[i].nnz; ++t) fr += E[i].v[t] * E[i].v[t];
                efrob[lev * ncol + k + 1] = sqrt(fr);
            }
        }
    }
    /* unscale: Lam <- W Lam W */
    for (int lev = 0; lev < nu; ++lev)
        for (int b = 0; b < nb; ++b) {
            int nbk = bptr[b + 1] - bptr[b];
            const int *rows = bidx + bptr[b];
            double *Lb = lam + (size_t)lev * lamsize + lamoff[b];
            for (int p = 0; p < nbk; ++p)
                for (int q = 0; q < nbk; ++q) Lb[p * nbk + q] *= w[rows[p]] * w[rows[q]];
        }
    for (int i = 0; i < N; ++i) { free(E[i].c); free(E[i].v); }
    free(E); free(Enew); free(blk_of); free(w);
    free(nptr); free(nblk); free(nloc); free(bnew);
    csr_free(&A);
    return 0;
}

static ora_casc *casc_alloc(const ora_hier *h, int kind, int nu) {
    ora_casc *c = xcalloc(1, sizeof(ora_casc));
    c->kind = kind; c->nu = nu;
    c->nlev = h->nlev > 1 ? h->nlev - 1 : 1;
    c->ncol = 1;
    for (int l = 0; l < c->nlev; ++l) {
        c->ncl[l] = kind == 1 ? h->ncol[l] : 1;
        if (c->ncl[l] > c->ncol) c->ncol = c->ncl[l];
    }
    for (int l = 0; l < c->nlev; ++l) {
        int nb = h->nb[l];
        c->lamoff[l] = xmalloc(sizeof(int64_t) * ((size_t)nb + 1));
        c->lamoff[l][0] = 0;
        for (int b = 0; b < nb; ++b) {
            int64_t nbk = h->bptr[l][b + 1] - h->bptr[l][b];
            c->lamoff[l][b + 1] = c->lamoff[l][b] + nbk * nbk;
        }
        c->lamsize[l] = c->lamoff[l][nb];
        c->lam[l] = xcalloc((size_t)nu * (size_t)c->lamsize[l], sizeof(double));
        c->efrob[l] = xcalloc((size_t)nu * c->ncl[l] + 1, sizeof(double));
    }
    return c;
}

void ora_casc_free(ora_casc *c) {
    if (!c) return;
    for (int l = 0; l < c->nlev; ++l) { free(c->lamoff[l]); free(c->lam[l]); free(c->efrob[l]); }
    free(c);
}

/* kind: 0 additive, 1 multiplicative (red-black).  Builds a cascade on every
 * level that has a smoother (all but the coarsest; a single-level hierarchy
 * gets one on its only level). */
/* spd != 0: every block of Lambda~ projected to the nearest symmetric
 * positive semidefinite matrix before the next step (for PCG). */
ora_casc *ora_casc_create_ex(const ora_hier *h, int kind, int nu, int prescale, int alpha, int spd) {
    ora_casc *c = casc_alloc(h, kind, nu);
    for (int l = 0; l < c->nlev; ++l) {
        if (cascade_level(h, l, kind, nu, prescale, alpha, spd, c->lamoff[l], c->lam[l], c->efrob[l]) != 0) {
            ora_casc_free(c);
            return NULL;
        }
    }
    return c;
}
/* ------------------------------------------------------ sketched setup
 * The sketched cascade of the concluding remarks (Sec. 4): each step
 * replaces min ||(I - Lam A) E_{l-1}||_F by min ||(I - Lam A) E_{l-1} S||_F
 * with an N x s sketching matrix S.  Carrying Y = E S (Y_0 = S), a step
 * solves, per block b, Lam~_b = argmin ||Y_b - Lam Z_b||_F with Z = A~ Y
 * (the same normal equations G = Z_b Z_b^T, C = Y_b Z_b^T as Algorithm 2)
 * and sets Y_b <- Y_b - Lam~_b Z_b; multiplicative: colour by colour, every
 * colour reading the state after the previous one (snapshot).  Prescaling
 * and unscaling as in the exact setup.  With exact_first, the first step
 * (multiplicative: its first colour, the one step whose residual is
 * E_0 = I) solves the unsketched problem (G = A~_b A~_b^T, C = A~_bb^T) and
 * Y becomes (I - Lam~_1 A~) S there (the hybrid the remarks suggest).
 *
 * S is Rademacher (entries +-1; its scale does not change Lam): entry (i, t)
 * of level l is the sign of the SplitMix64 output (Steele, Lea and Flood,
 * 2014) with counter c = l 2^48 + i s + t, i.e. of mix(seed + (c + 1) g),
 * g = 0x9E3779B97F4A7C15: +1 when its top bit is 0. */
static uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
static double rademacher(uint64_t seed, int l, int64_t i, int t, int s) {
    uint64_t c = ((uint64_t)l << 48) + (uint64_t)i * (uint64_t)s + (uint64_t)t;
    uint64_t z = sm64_mix(seed + (c + 1) * 0x9E3779B97F4A7C15ULL);
    return (z >> 63) ? -1.0 : 1.0;
}
double ora_rademacher(uint64_t seed, int l, int64_t i, int t, int s) { return rademacher(seed, l, i, t, s); }

static int sketch_level(const ora_hier *h, int l, int kind, int nu, int prescale, int s, uint64_t seed,
                        int exact_first, const int64_t *lamoff, double *lam) {
    const csr *A0 = &h->A[l];
    int N = A0->n, nb = h->nb[l];
    const int *bptr = h->bptr[l], *bidx = h->bidx[l];
    int ncol = kind == 1 ? h->ncol[l] : 1;
    int64_t lamsize = lamoff[nb];
    double *w = xmalloc(sizeof(double) * (size_t)N);
    if (prescale_weights(h, l, prescale, w) != 0) { free(w); return -1; }
    csr A;
    A.n = A.m = N;
    int64_t annz = A0->rp[N];
    A.rp = xmalloc(sizeof(int64_t) * ((size_t)N + 1));
    A.ci = xmalloc(sizeof(int) * (size_t)annz);
    A.v = xmalloc(sizeof(double) * (size_t)annz);
    memcpy(A.rp, A0->rp, sizeof(int64_t) * ((size_t)N + 1));
    memcpy(A.ci, A0->ci, sizeof(int) * (size_t)annz);
    for (int i = 0; i < N; ++i)
        for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p) A.v[p] = w[i] * A0->v[p] * w[A.ci[p]];
    double *Y = xmalloc(sizeof(double) * (size_t)N * s);
    double *Yn = xmalloc(sizeof(double) * (size_t)N * s);
    double *Z = xmalloc(sizeof(double) * (size_t)N * s);
    for (int64_t i = 0; i < N; ++i)
        for (int t = 0; t < s; ++t) Y[i * s + t] = rademacher(seed, l, i, t, s);
    memset(lam, 0, sizeof(double) * (size_t)nu * (size_t)lamsize);
    for (int step = 0; step < nu; ++step) {
        for (int k = 0; k < ncol; ++k) {
            /* Z = A~ Y */
            if (!(planted == PL_SKETCH_Z_ONCE && k > 0)) {
#pragma omp parallel for schedule(static)
            for (int i = 0; i < N; ++i)
                for (int t = 0; t < s; ++t) {
                    double z = 0.0;
                    for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p) z += A.v[p] * Y[(int64_t)A.ci[p] * s + t];
                    Z[(int64_t)i * s + t] = z;
                }
            }
            memcpy(Yn, Y, sizeof(double) * (size_t)N * s);
#pragma omp parallel for schedule(dynamic, 64)
            for (int b = 0; b < nb; ++b) {
                if (block_colour(h, l, kind, b) != k) continue;
                int nbk = bptr[b + 1] - bptr[b];
                const int *rows = bidx + bptr[b];
                double *G = xcalloc((size_t)nbk * nbk, sizeof(double));
                double *C = xcalloc((size_t)nbk * nbk, sizeof(double));
                if (step == 0 && k == 0 && exact_first) {
                    /* E_0 = I: R_b = A~_{b,:}, C_pq = A~(row_q, row_p) */
                    for (int p = 0; p < nbk; ++p)
                        for (int q = 0; q < nbk; ++q) {
                            double g = 0.0, c = 0.0;
                            int rp_ = rows[p], rq = rows[q];
                            for (int64_t u = A.rp[rp_]; u < A.rp[rp_ + 1]; ++u)
                                for (int64_t v = A.rp[rq]; v < A.rp[rq + 1]; ++v)
                                    if (A.ci[u] == A.ci[v]) g += A.v[u] * A.v[v];
                            if (planted == PL_SKETCH_FIRST_T) {
                                for (int64_t v = A.rp[rp_]; v < A.rp[rp_ + 1]; ++v)
                                    if (A.ci[v] == rq) c += A.v[v];
                            } else
                                for (int64_t v = A.rp[rq]; v < A.rp[rq + 1]; ++v)
                                    if (A.ci[v] == rp_) c += A.v[v];
                            G[p * nbk + q] = g; C[p * nbk + q] = c;
                        }
                } else {
                    for (int p = 0; p < nbk; ++p)
                        for (int q = 0; q < nbk; ++q) {
                            double g = 0.0, c = 0.0;
                            for (int t = 0; t < s; ++t) {
                                g += Z[(int64_t)rows[p] * s + t] * Z[(int64_t)rows[q] * s + t];
                                c += Y[(int64_t)rows[p] * s + t] * Z[(int64_t)rows[q] * s + t];
                            }
                            G[p * nbk + q] = g; C[p * nbk + q] = c;
                        }
                }
                double *Lb = lam + (size_t)step * lamsize + lamoff[b];
                ls_solve_block(G, C, nbk, Lb);
                for (int p = 0; p < nbk; ++p)
                    for (int t = 0; t < s; ++t) {
                        double y = Y[(int64_t)rows[p] * s + t];
                        for (int q = 0; q < nbk; ++q) y -= Lb[p * nbk + q] * Z[(int64_t)rows[q] * s + t];
                        Yn[(int64_t)rows[p] * s + t] = y;
                    }
                free(G); free(C);
            }
            if (planted != PL_SKETCH_STALE) { double *tmp = Y; Y = Yn; Yn = tmp; }
        }
    }
    for (int step = 0; step < nu; ++step)
        for (int b = 0; b < nb; ++b) {
            int nbk = bptr[b + 1] - bptr[b];
            const int *rows = bidx + bptr[b];
            double *Lb = lam + (size_t)step * lamsize + lamoff[b];
            for (int p = 0; p < nbk; ++p)
                for (int q = 0; q < nbk; ++q) Lb[p * nbk + q] *= w[rows[p]] * w[rows[q]];
        }
    free(Y); free(Yn); free(Z); free(w);
    csr_free(&A);
    return 0;
}

ora_casc *ora_casc_create_sketch(const ora_hier *h, int kind, int nu, int prescale, int s, uint64_t seed,
                                 int exact_first) {
    if (s < 1) return NULL;
    ora_casc *c = casc_alloc(h, kind, nu);
    for (int l = 0; l < c->nlev; ++l) {
        if (sketch_level(h, l, kind, nu, prescale, s, seed, exact_first, c->lamoff[l], c->lam[l]) != 0) {
            ora_casc_free(c);
            return NULL;
        }
    }
    return c;
}

ora_casc *ora_casc_create(const ora_hier *h, int kind, int nu, int prescale, int alpha) {
    return ora_casc_create_ex(h, kind, nu, prescale, alpha, 0);
}

/* A cascade with all Lambda = 0, to be filled by ora_casc_set_lambda. */
ora_casc *ora_casc_empty(const ora_hier *h, int kind, int nu) { return casc_alloc(h, kind, nu); }
int ora_casc_nlev(const ora_casc *c) { return c->nlev; }
int64_t ora_casc_lamsize(const ora_casc *c, int l) { return c->lamsize[l]; }
void ora_casc_lambda(const ora_casc *c, int l, double *out) {
    memcpy(out, c->lam[l], sizeof(double) * (size_t)c->nu * (size_t)c->lamsize[l]);
}
void ora_casc_set_lambda(ora_casc *c, int l, const double *in) {
    memcpy(c->lam[l], in, sizeof(double) * (size_t)c->nu * (size_t)c->lamsize[l]);
}
void ora_casc_efrob(const ora_casc *c, int l, double *out) {
    memcpy(out, c->efrob[l], sizeof(double) * ((size_t)c->nu * c->ncl[l] + 1));
}

/* ------------------------------------------------------------ smoother */
/* r = A x - b */
void ora_residual(const ora_hier *h, int l, const double *b, const double *x, double *r) {
    const csr *A = &h->A[l];
    csr_matvec(A, x, r);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < A->n; ++i) r[i] -= b[i];
}

/* One application of the depth-nu cascade on level l.
 * forward (reverse = 0): x <- x - Lam_{l,k} (A x - b), l = 1..nu, k = 1..chi
 *   (eq. fwda / fwdm); reverse: Lam_{nu-l+1, chi-k+1}^T in the same loop
 *   (eq. fwdar / fwdmr with the subscripts of the reverse propagator).
 * Within a colour every update reads the residual of the state before that
 * colour's step. */
void ora_smooth(const ora_hier *h, const ora_casc *c, int l, int reverse, const double *b, double *x) {
    int N = h->A[l].n, nb = h->nb[l];
    const int *bptr = h->bptr[l], *bidx = h->bidx[l];
    double *r = xmalloc(sizeof(double) * (size_t)N);
    for (int step = 0; step < c->nu; ++step) {
        int L = reverse && planted != PL_REVERSE_ORDER ? c->nu - 1 - step : step;
        for (int kk = 0; kk < c->ncl[l]; ++kk) {
            int K = reverse != (planted == PL_COLOUR_ORDER) ? c->ncl[l] - 1 - kk : kk;
            ora_residual(h, l, b, x, r);
            if (h->overlap[l] && c->kind == 0) {
                /* x -= diag(theta)^{-1} Theta^T Lambda Theta r (Sec. 3.6.2): the
                 * block corrections, then each node's average over its blocks */
                double *d = xmalloc(sizeof(double) * (size_t)bptr[nb]);
#pragma omp parallel for schedule(static)
                for (int bk = 0; bk < nb; ++bk) {
                    int nbk = bptr[bk + 1] - bptr[bk];
                    const int *rows = bidx + bptr[bk];
                    const double *Lb = c->lam[l] + (size_t)L * c->lamsize[l] + c->lamoff[l][bk];
                    for (int p = 0; p < nbk; ++p) {
                        double s = 0.0;
                        for (int q = 0; q < nbk; ++q)
                            s += (reverse ? Lb[q * nbk + p] : Lb[p * nbk + q]) * r[rows[q]];
                        d[bptr[bk] + p] = s;
                    }
                }
                int *nptr, *nblk, *nloc;
                node_blocks(h, l, &nptr, &nblk, &nloc);
#pragma omp parallel for schedule(static)
                for (int i = 0; i < N; ++i) {
                    double s = 0.0;
                    for (int u = nptr[i]; u < nptr[i + 1]; ++u) s += d[bptr[nblk[u]] + nloc[u]];
                    x[i] -= planted == PL_OVERLAP_SMOOTH_SUM ? s : s / (double)(nptr[i + 1] - nptr[i]);
                }
                free(d); free(nptr); free(nblk); free(nloc);
                continue;
            }
#pragma omp parallel for schedule(static)
            for (int bk = 0; bk < nb; ++bk) {
                if (block_colour(h, l, c->kind, bk) != K) continue;
                int nbk = bptr[bk + 1] - bptr[bk];
                const int *rows = bidx + bptr[bk];
                const double *Lb = c->lam[l] + (size_t)L * c->lamsize[l] + c->lamoff[l][bk];
                const int tr = reverse != (planted == PL_SMOOTH_T);
                for (int p = 0; p < nbk; ++p) {
                    double s = 0.0;
                    for (int q = 0; q < nbk; ++q)
                        s += (tr ? Lb[q * nbk + p] : Lb[p * nbk + q]) * r[rows[q]];
                    if (planted == PL_SMOOTH_SIGN) x[rows[p]] += s;
                    else x[rows[p]] -= s;
                }
            }
        }
    }
    free(r);
}

/* rc = R r (R = rscale P^T) */
void ora_restrict(const ora_hier *h, int l, const double *r, double *rc) { csr_matvec(&h->R[l], r, rc); }
/* x -= P xc */
void ora_prolong_correct(const ora_hier *h, int l, const double *xc, double *x) {
    const csr *P = &h->P[l];
#pragma omp parallel for schedule(static)
    for (int i = 0; i < P->n; ++i) {
        double s = 0.0;
        for (int64_t p = P->rp[i]; p < P->rp[i + 1]; ++p) s += P->v[p] * xc[P->ci[p]];
        if (planted == PL_PROLONG_SIGN) x[i] += s;
        else x[i] -= s;
    }
}
/* x = A_c^{-1} b on the coarsest level (dense Cholesky, LU if not SPD). */
void ora_coarse_solve(const ora_hier *h, const double *b, double *x) {
    for (int i = 0; i < h->cn; ++i) x[i] = b[i];
    if (h->cspd) chol_solve(h->cfac, h->cn, x);
    else lu_solve(h->cfac, h->cn, h->cpiv, x);
}

/* Algorithm 1, with mu_pre / mu_post applications of the cascade; the
 * pre-smoother is the reverse application when rf != 0. */
static void vcycle_rec(const ora_hier *h, const ora_casc *c, int l, int mu_pre, int mu_post, int rf,
                       const double *b, double *x) {
    if (l == h->nlev - 1) { ora_coarse_solve(h, b, x); return; }
    int N = h->A[l].n, Nc = h->A[l + 1].n;
    for (int m = 0; m < mu_pre; ++m) ora_smooth(h, c, l, rf && planted != PL_RF_FORWARD ? 1 : 0, b, x);
    double *r = xmalloc(sizeof(double) * (size_t)N);
    double *rc = xmalloc(sizeof(double) * (size_t)Nc);
    double *xc = xcalloc((size_t)Nc, sizeof(double));
    ora_residual(h, l, b, x, r);
    ora_restrict(h, l, r, rc);
    vcycle_rec(h, c, l + 1, mu_pre, mu_post, rf, rc, xc);
    ora_prolong_correct(h, l, xc, x);
    for (int m = 0; m < mu_post; ++m) ora_smooth(h, c, l, 0, b, x);
    free(r); free(rc); free(xc);
}
void ora_vcycle(const ora_hier *h, const ora_casc *c, int mu_pre, int mu_post, int rf, const double *b, double *x) {
    vcycle_rec(h, c, 0, mu_pre, mu_post, rf, b, x);
}

static double nrm2(const double *x, int n) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += x[i] * x[i];
    return sqrt(s);
}

/* Stationary iteration x <- V(x, b) (method 0) or left-preconditioned
 * restarted GMRES(restart) with M = V(0, .) (method 1, Sec. 3.1).
 * Stops when ||b - A x||_2 / ||b||_2 <= tol.  hist[0..*nhist-1] receives
 * the relative true residuals (stationary) or the relative preconditioned
 * residual estimates ||M(b - A x_i)|| / ||M b|| (GMRES); returns the number
 * of iterations (V-cycle applications after the initial one for GMRES), or
 * -1 when maxit is reached without convergence. */
int ora_solve(const ora_hier *h, const ora_casc *c, int method, int mu_pre, int mu_post, int rf,
              double tol, int maxit, int restart, const double *b, double *x, double *hist, int *nhist,
              double *final_rel) {
    int N = h->A[0].n;
    double nb = nrm2(b, N);
    double *r = xmalloc(sizeof(double) * (size_t)N);
    int nh = 0, it = 0, conv = 0;
    if (nb == 0.0) {
        for (int i = 0; i < N; ++i) x[i] = 0.0;
        if (final_rel) *final_rel = 0.0;
        *nhist = 0; free(r); return 0;
    }
    if (method == 0) {
        ora_residual(h, 0, b, x, r);
        double rel = nrm2(r, N) / nb;
        hist[nh++] = rel;
        while (rel > tol && it < maxit) {
            ora_vcycle(h, c, mu_pre, mu_post, rf, b, x);
            ++it;
            ora_residual(h, 0, b, x, r);
            rel = nrm2(r, N) / nb;
            hist[nh++] = rel;
        }
        conv = rel <= tol;
        if (final_rel) *final_rel = rel;
    } else if (method == 3) {
        /* preconditioned conjugate gradient with M = V(0, .) (SM "On
         * preconditioned conjugate gradient"; M must be SPD for it to
         * converge); history: ||b - A x_k|| / ||b|| of the recurrence */
        double *z = xmalloc(sizeof(double) * (size_t)N), *pv = xmalloc(sizeof(double) * (size_t)N);
        double *q = xmalloc(sizeof(double) * (size_t)N);
        ora_residual(h, 0, b, x, r);
        for (int i = 0; i < N; ++i) r[i] = -r[i];
        double rel = nrm2(r, N) / nb;
        hist[nh++] = rel;
        for (int i = 0; i < N; ++i) z[i] = 0.0;
        ora_vcycle(h, c, mu_pre, mu_post, rf, r, z);
        double rz = 0.0;
        for (int i = 0; i < N; ++i) { pv[i] = z[i]; rz += r[i] * z[i]; }
        while (rel > tol && it < maxit) {
            csr_matvec(&h->A[0], pv, q);
            double pq = 0.0;
            for (int i = 0; i < N; ++i) pq += pv[i] * q[i];
            double alpha = rz / pq;
            for (int i = 0; i < N; ++i) { x[i] += alpha * pv[i]; r[i] -= alpha * q[i]; }
            ++it;
            rel = nrm2(r, N) / nb;
            hist[nh++] = rel;
            if (!(rel > tol)) break;
            for (int i = 0; i < N; ++i) z[i] = 0.0;
            ora_vcycle(h, c, mu_pre, mu_post, rf, r, z);
            double rz1 = 0.0;
            for (int i = 0; i < N; ++i) rz1 += r[i] * z[i];
            double beta = planted == PL_PCG_BETA ? rz / rz1 : rz1 / rz;
            rz = rz1;
            for (int i = 0; i < N; ++i) pv[i] = z[i] + beta * pv[i];
        }
        /* the true residual decides */
        ora_residual(h, 0, b, x, r);
        rel = nrm2(r, N) / nb;
        conv = rel <= tol;
        if (final_rel) *final_rel = rel;
        free(z); free(pv); free(q);
    } else if (method == 2) {
        /* Right-preconditioned restarted GMRES (Sec. 3.1 with the cycle
         * applied on the right): x_k minimises the TRUE residual
         * ||b - A x|| over x_0 + span{Z_0..Z_{k-1}}, Z_j = M V_j, with V an
         * orthonormal (modified Gram-Schmidt) basis of K_k(A M, r_0).  The
         * Givens estimate |g_{j+1}| is ||b - A x_j|| itself, so the inner
         * loop stops on the true residual. */
        int m = restart;
        double *V = xmalloc(sizeof(double) * (size_t)N * (m + 1));
        double *Z = xmalloc(sizeof(double) * (size_t)N * m);
        double *H = xcalloc((size_t)(m + 1) * m, sizeof(double));
        double *cs = xmalloc(sizeof(double) * m), *sn = xmalloc(sizeof(double) * m);
        double *g = xmalloc(sizeof(double) * (m + 1)), *y = xmalloc(sizeof(double) * m);
        double rel = 1.0;
        for (;;) {
            ora_residual(h, 0, b, x, r); /* r = A x - b */
            double beta = nrm2(r, N);
            rel = beta / nb;
            if (nh == 0) hist[nh++] = rel;
            if (rel <= tol || it >= maxit) break;
            for (int i = 0; i < N; ++i) V[i] = -r[i] / beta;
            for (int i = 0; i <= m; ++i) g[i] = 0.0;
            g[0] = beta;
            int j;
            for (j = 0; j < m && it < maxit; ++j) {
                /* z_j = M v_j, w = A z_j */
                double *z = Z + (size_t)j * N;
                for (int i = 0; i < N; ++i) z[i] = 0.0;
                ora_vcycle(h, c, mu_pre, mu_post, rf, V + (size_t)j * N, z);
                ++it;
                double *w = V + (size_t)(j + 1) * N;
                csr_matvec(&h->A[0], z, w);
                for (int i = 0; i <= j; ++i) {
                    double d = 0.0;
                    for (int q = 0; q < N; ++q) d += w[q] * V[(size_t)i * N + q];
                    H[i * m + j] = d;
                    for (int q = 0; q < N; ++q) w[q] -= d * V[(size_t)i * N + q];
                }
                double hn = nrm2(w, N);
                H[(j + 1) * m + j] = hn;
                if (hn > 0.0) for (int q = 0; q < N; ++q) w[q] /= hn;
                for (int i = 0; i < j; ++i) {
                    double a = H[i * m + j], bb = H[(i + 1) * m + j];
                    H[i * m + j] = cs[i] * a + sn[i] * bb;
                    H[(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
                }
                double a = H[j * m + j], bb = H[(j + 1) * m + j];
                double d = sqrt(a * a + bb * bb);
                cs[j] = d > 0 ? a / d : 1.0; sn[j] = d > 0 ? bb / d : 0.0;
                H[j * m + j] = d; H[(j + 1) * m + j] = 0.0;
                g[j + 1] = -sn[j] * g[j];
                g[j] = cs[j] * g[j];
                hist[nh++] = fabs(g[j + 1]) / nb;
                if (fabs(g[j + 1]) <= tol * nb || hn == 0.0) { ++j; break; }
            }
            /* x += Z y, H y = g */
            for (int i = j - 1; i >= 0; --i) {
                double s = g[i];
                for (int k = i + 1; k < j; ++k) s -= H[i * m + k] * y[k];
                y[i] = s / H[i * m + i];
            }
            const double *U = planted == PL_RIGHT_UPDATE_V ? V : Z;
            for (int i = 0; i < j; ++i)
                for (int q = 0; q < N; ++q) x[q] += y[i] * U[(size_t)i * N + q];
        }
        conv = rel <= tol;
        if (final_rel) *final_rel = rel;
        free(V); free(Z); free(H); free(cs); free(sn); free(g); free(y);
    } else {
        int m = restart;
        double *V = xmalloc(sizeof(double) * (size_t)N * (m + 1));
        double *H = xcalloc((size_t)(m + 1) * m, sizeof(double));
        double *cs = xmalloc(sizeof(double) * m), *sn = xmalloc(sizeof(double) * m);
        double *g = xmalloc(sizeof(double) * (m + 1)), *y = xmalloc(sizeof(double) * m);
        double *t = xmalloc(sizeof(double) * (size_t)N);
        /* ||M b|| */
        for (int i = 0; i < N; ++i) t[i] = 0.0;
        ora_vcycle(h, c, mu_pre, mu_post, rf, b, t);
        double nmb = nrm2(t, N);
        double rel = 1.0;
        for (;;) {
            /* z = M (b - A x) */
            ora_residual(h, 0, b, x, r);
            for (int i = 0; i < N; ++i) r[i] = -r[i];
            ora_residual(h, 0, b, x, t);
            rel = nrm2(t, N) / nb;
            if (rel <= tol || it >= maxit) break;
            for (int i = 0; i < N; ++i) t[i] = 0.0;
            ora_vcycle(h, c, mu_pre, mu_post, rf, r, t);
            double beta = nrm2(t, N);
            if (nh == 0) hist[nh++] = beta / nmb;
            for (int i = 0; i < N; ++i) V[i] = t[i] / beta;
            for (int i = 0; i <= m; ++i) g[i] = 0.0;
            g[0] = beta;
            int j;
            for (j = 0; j < m && it < maxit; ++j) {
                /* w = M A v_j */
                csr_matvec(&h->A[0], V + (size_t)j * N, r);
                double *w = V + (size_t)(j + 1) * N;
                for (int i = 0; i < N; ++i) w[i] = 0.0;
                ora_vcycle(h, c, mu_pre, mu_post, rf, r, w);
                ++it;
                /* modified Gram-Schmidt */
                for (int i = 0; i <= j; ++i) {
                    double d = 0.0;
                    for (int q = 0; q < N; ++q) d += w[q] * V[(size_t)i * N + q];
                    H[i * m + j] = d;
                    for (int q = 0; q < N; ++q) w[q] -= d * V[(size_t)i * N + q];
                }
                double hn = nrm2(w, N);
                H[(j + 1) * m + j] = hn;
                if (hn > 0.0) for (int q = 0; q < N; ++q) w[q] /= hn;
                /* Givens rotations */
                for (int i = 0; i < j; ++i) {
                    double a = H[i * m + j], bb = H[(i + 1) * m + j];
                    H[i * m + j] = cs[i] * a + sn[i] * bb;
                    H[(i + 1) * m + j] = (planted == PL_GIVENS_SIGN ? sn[i] : -sn[i]) * a + cs[i] * bb;
                }
                double a = H[j * m + j], bb = H[(j + 1) * m + j];
                double d = sqrt(a * a + bb * bb);
                cs[j] = d > 0 ? a / d : 1.0; sn[j] = d > 0 ? bb / d : 0.0;
                H[j * m + j] = d; H[(j + 1) * m + j] = 0.0;
                g[j + 1] = -sn[j] * g[j];
                g[j] = cs[j] * g[j];
                hist[nh++] = fabs(g[j + 1]) / nmb;
                if (fabs(g[j + 1]) <= tol * nmb || hn == 0.0) { ++j; break; }
            }
            /* x += V y, H y = g */
            for (int i = j - 1; i >= 0; --i) {
                double s = g[i];
                for (int k = i + 1; k < j; ++k) s -= H[i * m + k] * y[k];
                y[i] = s / H[i * m + i];
            }
            for (int i = 0; i < j; ++i)
                for (int q = 0; q < N; ++q) x[q] += y[i] * V[(size_t)i * N + q];
        }
        conv = rel <= tol;
        if (final_rel) *final_rel = rel;
        free(V); free(H); free(cs); free(sn); free(g); free(y); free(t);
    }
    *nhist = nh;
    free(r);
    return conv ? it : -1;
}
