/*
 * olu.c -- the oracle's own sparse direct solver (TEST INFRASTRUCTURE ONLY: called from
 * oracle/sparse_lu.py, which only tests/, the smoke check and the benchmark's CPU baseline
 * import).  Nothing here is shared with the CUDA library.
 *
 * Every G_k^{-1} b of the ER step (Alg. 2 "LU_decompose(G_k)", Algorithm 1 "Solve
 * -G w = C v_j") goes through this factorisation:
 *   - ordering: minimum degree on the pattern of A + A^T (Tinney-Walker scheme 2) over a
 *     quotient graph: an eliminated node becomes an "element" holding its fill clique, and
 *     the degree of a variable is bounded from its variable neighbours and the cliques of its
 *     elements (the approximate degree of Amestoy, Davis and Duff);
 *   - factorisation: left-looking LU with threshold partial pivoting (Gilbert & Peierls,
 *     1988): column k of L and U comes from one sparse triangular solve L x = A(:, q_k)
 *     whose nonzero pattern is the reach of A(:, q_k) in the graph of L (depth-first search,
 *     topological order), then a pivot choice that keeps the diagonal entry when
 *     |x_diag| >= tau * max |x|;
 *   - solve: P A Q = L U, x = Q U^{-1} L^{-1} P b.
 * Plain C99, no intrinsics; portable between x86-64 and aarch64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OLU_OK 0
#define OLU_SINGULAR 1
#define OLU_NOMEM 2
#define OLU_INVALID 3

typedef struct {
  int32_t* a;
  int32_t len, cap;
} ivec;

static int iv_push(ivec* v, int32_t x) {
  if (v->len == v->cap) {
    int32_t nc = v->cap ? 2 * v->cap : 4;
    int32_t* na = (int32_t*)realloc(v->a, (size_t)nc * sizeof(int32_t));
    if (!na) return 0;
    v->a = na;
    v->cap = nc;
  }
  v->a[v->len++] = x;
  return 1;
}

static void iv_free(ivec* v) {
  free(v->a);
  v->a = NULL;
  v->len = v->cap = 0;
}

/* ---------------------------------------------------------------------------------------
 * Minimum-degree ordering.  Ap/Ai: CSC (or CSR: the pattern is symmetrised) of an n x n
 * matrix; perm[k] receives the k-th eliminated node.  Returns OLU_OK or OLU_NOMEM.
 * Degrees after an elimination are the upper bound of approximate minimum degree
 * (Amestoy, Davis & Duff, SIAM J. Matrix Anal. Appl. 17, 1996): for a variable v of the new
 * element p,  d(v) <= min(remaining - 1, d_old(v) + |L_p| - 1,
 *                         |A_v| + |L_p| - 1 + sum_{e in E_v, e != p} |L_e \ L_p|),
 * where |L_e \ L_p| is found for every element in one pass over the new clique.
 * ------------------------------------------------------------------------------------- */
enum { MD_VAR = 0, MD_ELEM = 1, MD_DEAD = 2 };

int olu_order(int32_t n, const int32_t* Ap, const int32_t* Ai, int32_t* perm) {
  if (n < 0) return OLU_INVALID;
  if (n == 0) return OLU_OK;
  int rc = OLU_NOMEM;
  ivec* avar = (ivec*)calloc((size_t)n, sizeof(ivec));    /* variable neighbours */
  ivec* elem = (ivec*)calloc((size_t)n, sizeof(ivec));    /* adjacent elements */
  ivec* clq = (ivec*)calloc((size_t)n, sizeof(ivec));     /* element cliques */
  int32_t* st = (int32_t*)calloc((size_t)n, sizeof(int32_t));
  int32_t* deg = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  int32_t* head = (int32_t*)malloc((size_t)(n + 1) * sizeof(int32_t));
  int32_t* nxt = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  int32_t* prv = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  int64_t* mark = (int64_t*)calloc((size_t)n, sizeof(int64_t));
  int64_t* mark2 = (int64_t*)calloc((size_t)n, sizeof(int64_t));
  int32_t* ext = (int32_t*)calloc((size_t)n, sizeof(int32_t));   /* |L_e \ L_p| */
  int64_t stamp = 0, stamp2 = 0;
  ivec lp = {0};
  if (!avar || !elem || !clq || !st || !deg || !head || !nxt || !prv || !mark || !mark2 ||
      !ext)
    goto done;
  /* symmetric adjacency without self loops, duplicates removed with a marker */
  for (int32_t j = 0; j < n; ++j)
    for (int32_t e = Ap[j]; e < Ap[j + 1]; ++e) {
      int32_t i = Ai[e];
      if (i == j || i < 0 || i >= n) continue;
      if (!iv_push(&avar[i], j) || !iv_push(&avar[j], i)) goto done;
    }
  for (int32_t v = 0; v < n; ++v) {
    ++stamp;
    int32_t w = 0;
    for (int32_t t = 0; t < avar[v].len; ++t) {
      int32_t u = avar[v].a[t];
      if (mark[u] == stamp) continue;
      mark[u] = stamp;
      avar[v].a[w++] = u;
    }
    avar[v].len = w;
    deg[v] = w;
  }
  /* degree buckets (doubly linked lists) */
  for (int32_t d = 0; d <= n; ++d) head[d] = -1;
#define BUCKET_IN(v)                                   \
  do {                                                 \
    int32_t d_ = deg[v] < n ? deg[v] : n;              \
    nxt[v] = head[d_];                                 \
    prv[v] = -1;                                       \
    if (head[d_] >= 0) prv[head[d_]] = (v);            \
    head[d_] = (v);                                    \
  } while (0)
#define BUCKET_OUT(v)                                  \
  do {                                                 \
    int32_t d_ = deg[v] < n ? deg[v] : n;              \
    if (prv[v] >= 0) nxt[prv[v]] = nxt[v];             \
    else head[d_] = nxt[v];                            \
    if (nxt[v] >= 0) prv[nxt[v]] = prv[v];             \
  } while (0)
  for (int32_t v = n - 1; v >= 0; --v) BUCKET_IN(v);
  int32_t dmin = 0;
  for (int32_t k = 0; k < n; ++k) {
    while (dmin <= n && head[dmin] < 0) ++dmin;
    int32_t p = head[dmin];
    BUCKET_OUT(p);
    perm[k] = p;
    /* clique of the new element: variable neighbours and the cliques of p's elements */
    ++stamp;
    mark[p] = stamp;
    lp.len = 0;
    for (int32_t t = 0; t < avar[p].len; ++t) {
      int32_t u = avar[p].a[t];
      if (st[u] != MD_VAR || mark[u] == stamp) continue;
      mark[u] = stamp;
      if (!iv_push(&lp, u)) goto done;
    }
    for (int32_t t = 0; t < elem[p].len; ++t) {
      int32_t e = elem[p].a[t];
      if (st[e] != MD_ELEM) continue;
      for (int32_t s = 0; s < clq[e].len; ++s) {
        int32_t u = clq[e].a[s];
        if (st[u] != MD_VAR || mark[u] == stamp) continue;
        mark[u] = stamp;
        if (!iv_push(&lp, u)) goto done;
      }
      st[e] = MD_DEAD;           /* absorbed into p's element */
      iv_free(&clq[e]);
    }
    st[p] = MD_ELEM;
    iv_free(&avar[p]);
    iv_free(&elem[p]);
    for (int32_t t = 0; t < lp.len; ++t)
      if (!iv_push(&clq[p], lp.a[t])) goto done;
    /* update the neighbours of p: drop absorbed elements, prune variable neighbours now
     * covered by p's clique; then |L_e \ L_p| for every other element next to the clique */
    for (int32_t t = 0; t < lp.len; ++t) {
      int32_t v = lp.a[t];
      int32_t w = 0;
      for (int32_t s = 0; s < elem[v].len; ++s) {
        int32_t e = elem[v].a[s];
        if (st[e] == MD_ELEM) elem[v].a[w++] = e;
      }
      elem[v].len = w;
      w = 0;
      for (int32_t s = 0; s < avar[v].len; ++s) {
        int32_t u = avar[v].a[s];
        if (st[u] == MD_VAR && mark[u] != stamp) avar[v].a[w++] = u;
      }
      avar[v].len = w;
    }
    ++stamp2;
    for (int32_t t = 0; t < lp.len; ++t) {
      int32_t v = lp.a[t];
      for (int32_t s = 0; s < elem[v].len; ++s) {
        int32_t e = elem[v].a[s];
        if (mark2[e] != stamp2) { mark2[e] = stamp2; ext[e] = clq[e].len; }
        ext[e] -= 1;   /* v lies in both L_e and L_p */
      }
    }
    const int32_t remaining = n - 1 - k;
    for (int32_t t = 0; t < lp.len; ++t) {
      int32_t v = lp.a[t];
      int64_t bound = (int64_t)avar[v].len + lp.len - 1;
      for (int32_t s = 0; s < elem[v].len; ++s) bound += ext[elem[v].a[s]];
      int64_t d = remaining - 1;
      if ((int64_t)deg[v] + lp.len - 1 < d) d = (int64_t)deg[v] + lp.len - 1;
      if (bound < d) d = bound;
      if (d < 0) d = 0;
      if (!iv_push(&elem[v], p)) goto done;
      BUCKET_OUT(v);
      deg[v] = (int32_t)d;
      BUCKET_IN(v);
      if (deg[v] < dmin) dmin = deg[v];
    }
  }
#undef BUCKET_IN
#undef BUCKET_OUT
  rc = OLU_OK;
done:
  if (avar) for (int32_t v = 0; v < n; ++v) iv_free(&avar[v]);
  if (elem) for (int32_t v = 0; v < n; ++v) iv_free(&elem[v]);
  if (clq) for (int32_t v = 0; v < n; ++v) iv_free(&clq[v]);
  free(avar); free(elem); free(clq); free(st); free(deg); free(head); free(nxt); free(prv);
  free(mark); free(mark2); free(ext);
  iv_free(&lp);
  return rc;
}

/* ---------------------------------------------------------------------------------------
 * Left-looking LU with threshold partial pivoting.
 * ------------------------------------------------------------------------------------- */
typedef struct {
  int32_t n;
  int64_t* Lp;   /* n + 1 */
  int32_t* Li;   /* original row indices of the strictly lower part of L (unit diagonal) */
  double* Lx;
  int64_t* Up;   /* n + 1 */
  int32_t* Ui;   /* pivot positions (< k) of column k of U; the diagonal comes last */
  double* Ux;
  int32_t* pinv; /* pinv[original row] = pivot position */
  int32_t* prow; /* prow[pivot position] = original row */
  int32_t* q;    /* q[k] = original column of factor column k */
  int64_t lcap, ucap;
} olu_t;

void olu_free(olu_t* F) {
  if (!F) return;
  free(F->Lp); free(F->Li); free(F->Lx); free(F->Up); free(F->Ui); free(F->Ux);
  free(F->pinv); free(F->prow); free(F->q);
  free(F);
}

static int grow_l(olu_t* F, int64_t need) {
  if (need <= F->lcap) return 1;
  int64_t nc = F->lcap * 2 > need ? F->lcap * 2 : need;
  int32_t* ni = (int32_t*)realloc(F->Li, (size_t)nc * sizeof(int32_t));
  if (!ni) return 0;
  F->Li = ni;
  double* nx = (double*)realloc(F->Lx, (size_t)nc * sizeof(double));
  if (!nx) return 0;
  F->Lx = nx;
  F->lcap = nc;
  return 1;
}

static int grow_u(olu_t* F, int64_t need) {
  if (need <= F->ucap) return 1;
  int64_t nc = F->ucap * 2 > need ? F->ucap * 2 : need;
  int32_t* ni = (int32_t*)realloc(F->Ui, (size_t)nc * sizeof(int32_t));
  if (!ni) return 0;
  F->Ui = ni;
  double* nx = (double*)realloc(F->Ux, (size_t)nc * sizeof(double));
  if (!nx) return 0;
  F->Ux = nx;
  F->ucap = nc;
  return 1;
}

/* Factor the n x n CSC matrix (Ap, Ai, Ax) with column order q (NULL: natural) and pivot
 * threshold tau in (0, 1].  *out receives the factorisation.  Returns OLU_SINGULAR when a
 * column has no nonzero pivot candidate. */
int olu_factor(int32_t n, const int32_t* Ap, const int32_t* Ai, const double* Ax,
               const int32_t* q, double tau, olu_t** out) {
  *out = NULL;
  if (n < 0 || !(tau > 0.0) || tau > 1.0) return OLU_INVALID;
  olu_t* F = (olu_t*)calloc(1, sizeof(olu_t));
  if (!F) return OLU_NOMEM;
  F->n = n;
  int64_t nnzA = n > 0 ? Ap[n] : 0;
  F->lcap = F->ucap = 4 * nnzA + n + 16;
  F->Lp = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  F->Up = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  F->Li = (int32_t*)malloc((size_t)F->lcap * sizeof(int32_t));
  F->Lx = (double*)malloc((size_t)F->lcap * sizeof(double));
  F->Ui = (int32_t*)malloc((size_t)F->ucap * sizeof(int32_t));
  F->Ux = (double*)malloc((size_t)F->ucap * sizeof(double));
  F->pinv = (int32_t*)malloc((size_t)(n + 1) * sizeof(int32_t));
  F->prow = (int32_t*)malloc((size_t)(n + 1) * sizeof(int32_t));
  F->q = (int32_t*)malloc((size_t)(n + 1) * sizeof(int32_t));
  double* x = (double*)calloc((size_t)n + 1, sizeof(double));
  int32_t* reach = (int32_t*)malloc((size_t)(n + 1) * sizeof(int32_t));   /* topological */
  int32_t* stk = (int32_t*)malloc((size_t)(n + 1) * sizeof(int32_t));     /* DFS nodes */
  int64_t* pos = (int64_t*)malloc((size_t)(n + 1) * sizeof(int64_t));     /* DFS positions */
  int32_t* seen = (int32_t*)malloc((size_t)(n + 1) * sizeof(int32_t));
  int rc = OLU_NOMEM;
  if (!F->Lp || !F->Up || !F->Li || !F->Lx || !F->Ui || !F->Ux || !F->pinv || !F->prow ||
      !F->q || !x || !reach || !stk || !pos || !seen)
    goto fail;
  for (int32_t i = 0; i < n; ++i) {
    F->pinv[i] = -1;
    seen[i] = -1;
    F->q[i] = q ? q[i] : i;
  }
  for (int32_t k = 0; k < n; ++k) {
    const int32_t j = F->q[k];
    if (j < 0 || j >= n) { rc = OLU_INVALID; goto fail; }
    /* reach of A(:, j) in the graph of L: depth-first search from every row of the
     * column; an edge leads from a pivoted row (position p) to the rows of L(:, p) */
    int32_t top = n;   /* reach[top..n) in topological order */
    for (int32_t e = Ap[j]; e < Ap[j + 1]; ++e) {
      int32_t r0 = Ai[e];
      if (seen[r0] == k) continue;
      int32_t sp = 0;
      stk[0] = r0;
      seen[r0] = k;
      pos[0] = -1;
      while (sp >= 0) {
        int32_t r = stk[sp];
        int32_t pr = F->pinv[r];
        if (pos[sp] < 0) pos[sp] = pr >= 0 ? F->Lp[pr] : 0;
        int pushed = 0;
        if (pr >= 0) {
          int64_t end = F->Lp[pr + 1];
          while (pos[sp] < end) {
            int32_t c = F->Li[pos[sp]++];
            if (seen[c] == k) continue;
            seen[c] = k;
            stk[++sp] = c;
            pos[sp] = -1;
            pushed = 1;
            break;
          }
        }
        if (!pushed) {
          reach[--top] = r;   /* finished: prepend (reverse postorder) */
          --sp;
        }
      }
    }
    /* numeric sparse triangular solve in topological order */
    for (int32_t e = Ap[j]; e < Ap[j + 1]; ++e) x[Ai[e]] += Ax[e];
    for (int32_t t = top; t < n; ++t) {
      int32_t r = reach[t];
      int32_t pr = F->pinv[r];
      if (pr < 0) continue;
      double xr = x[r];
      for (int64_t e = F->Lp[pr]; e < F->Lp[pr + 1]; ++e) x[F->Li[e]] -= F->Lx[e] * xr;
    }
    /* pivot among the rows not yet pivotal: the diagonal row j when it is large enough */
    double amax = -1.0;
    int32_t ipiv = -1;
    for (int32_t t = top; t < n; ++t) {
      int32_t r = reach[t];
      if (F->pinv[r] >= 0) continue;
      double a = fabs(x[r]);
      if (a > amax) { amax = a; ipiv = r; }
    }
    if (ipiv < 0 || !(amax > 0.0) || !isfinite(amax)) { rc = OLU_SINGULAR; goto fail; }
    if (seen[j] == k && F->pinv[j] < 0 && fabs(x[j]) >= tau * amax) ipiv = j;
    const double piv = x[ipiv];
    /* column k of U (pivotal rows, diagonal last) and of L (the rest, divided) */
    int64_t un = F->Up[k], ln = F->Lp[k];
    if (!grow_u(F, un + (n - top) + 1) || !grow_l(F, ln + (n - top) + 1)) goto fail;
    for (int32_t t = top; t < n; ++t) {
      int32_t r = reach[t];
      int32_t pr = F->pinv[r];
      if (pr >= 0) {
        F->Ui[un] = pr;
        F->Ux[un++] = x[r];
      } else if (r != ipiv) {
        F->Li[ln] = r;
        F->Lx[ln++] = x[r] / piv;
      }
      x[r] = 0.0;
    }
    F->Ui[un] = k;
    F->Ux[un++] = piv;
    F->Up[k + 1] = un;
    F->Lp[k + 1] = ln;
    F->pinv[ipiv] = k;
    F->prow[k] = ipiv;
  }
  free(x); free(reach); free(stk); free(pos); free(seen);
  *out = F;
  return OLU_OK;
fail:
  free(x); free(reach); free(stk); free(pos); free(seen);
  olu_free(F);
  return rc;
}

/* x = A^{-1} b for nrhs right-hand sides (column-major, stride n); b and x may alias.
 * work: n doubles. */
void olu_solve(const olu_t* F, int32_t nrhs, const double* b, double* x, double* work) {
  const int32_t n = F->n;
  for (int32_t c = 0; c < nrhs; ++c) {
    const double* bc = b + (int64_t)c * n;
    double* xc = x + (int64_t)c * n;
    /* forward: L y = P b, kept in original row indexing, y_k read at row prow[k] */
    for (int32_t i = 0; i < n; ++i) work[i] = bc[i];
    for (int32_t k = 0; k < n; ++k) {
      double yk = work[F->prow[k]];
      for (int64_t e = F->Lp[k]; e < F->Lp[k + 1]; ++e) work[F->Li[e]] -= F->Lx[e] * yk;
    }
    /* y in pivot order, then backward: U z = y (diagonal is the last entry of a column) */
    for (int32_t k = 0; k < n; ++k) xc[k] = work[F->prow[k]];
    for (int32_t k = n - 1; k >= 0; --k) {
      int64_t d = F->Up[k + 1] - 1;
      double zk = xc[k] / F->Ux[d];
      xc[k] = zk;
      for (int64_t e = F->Up[k]; e < d; ++e) xc[F->Ui[e]] -= F->Ux[e] * zk;
    }
    /* x(q_k) = z_k */
    for (int32_t k = 0; k < n; ++k) work[F->q[k]] = xc[k];
    for (int32_t i = 0; i < n; ++i) xc[i] = work[i];
  }
}

int64_t olu_nnz_l(const olu_t* F) { return F->n ? F->Lp[F->n] + F->n : 0; }
int64_t olu_nnz_u(const olu_t* F) { return F->n ? F->Up[F->n] : 0; }

/* Export the factors for checking P A Q = L U: L (strictly lower part, rows as pivot
 * positions), U (with diagonal), both CSC over factor columns; and prow, q.  Arrays must
 * hold olu_nnz_l - n (L) and olu_nnz_u (U) entries. */
void olu_export(const olu_t* F, int64_t* Lp, int32_t* Li, double* Lx, int64_t* Up,
                int32_t* Ui, double* Ux, int32_t* prow, int32_t* q) {
  const int32_t n = F->n;
  for (int32_t k = 0; k <= n; ++k) { Lp[k] = F->Lp[k]; Up[k] = F->Up[k]; }
  for (int64_t e = 0; e < F->Lp[n]; ++e) { Li[e] = F->pinv[F->Li[e]]; Lx[e] = F->Lx[e]; }
  for (int64_t e = 0; e < F->Up[n]; ++e) { Ui[e] = F->Ui[e]; Ux[e] = F->Ux[e]; }
  for (int32_t k = 0; k < n; ++k) { prow[k] = F->prow[k]; q[k] = F->q[k]; }
}
