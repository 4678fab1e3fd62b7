/*
 * fd_oracle.c -- FP64 CPU oracle for the SOR stress-majorization layout method
 * of Wang & Wang, "A Fast Successive Over-Relaxation Algorithm for
 * Force-Directed Network Graph Drawing" (Sci. China Inf. Sci. 55:677, 2012).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct reference
 * that the CUDA path is checked against.  Only the test suite, the smoke check
 * and the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or constant with the CUDA library, and it never includes or
 * links anything from the package.
 *
 * Everything is plain double-precision C: explicit loops over vertices and
 * vertex pairs, no blocking, no fusion.  Positions X are row-major [n][dim].
 * Ideal distances D are a dense row-major [n][n] double matrix.
 *
 * Notation (Section 2 of the paper):
 *   stress  f(X)   = sum_{i<j} w_ij (||x_i - x_j|| - d_ij)^2          Eq. (1)
 *   weights w_ij   = d_ij^{-2}                                        Sec. 5.1
 *   L^W   : l_ij = -w_ij (i != j), l_ii = -sum_{k != i} l_ik           Prop. 2.1
 *   L^Y   : l_ij = -w_ij d_ij / ||y_i - y_j|| (i != j, y_i != y_j),
 *           l_ij = 0 if y_i == y_j, diagonal = negative off-diagonal row sum
 *   majorization step: L^W X^{k+1} = L^{X^k} X^k                      Eq. (2-5)
 *
 * Parity status of each function is stated in oracle/oracle.py's header.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_DISCONNECTED 3
#define ORC_ERR_OOM 8

/* ------------------------------------------------------------------------ */
/* Ideal distances d_ij: graph-theoretic shortest-path lengths.               */
/* The paper calls d_ij the "predefined ideal distance" (Sec. 2, Eq. (1)) and  */
/* follows Gansner et al., whose d_ij is the shortest-path distance; edges     */
/* of weighted graphs carry lengths (railway net, Sec. 5.4).                  */
/* ------------------------------------------------------------------------ */

/* Breadth-first search from src over an unweighted CSR graph.
 * dist[v] = number of edges on a shortest src-v path, -1 if unreachable.
 * queue must hold n ints. */
void orc_bfs(int n, const int *row_ptr, const int *col_idx, int src, int *dist,
             int *queue) {
  for (int v = 0; v < n; ++v) dist[v] = -1;
  int head = 0, tail = 0;
  dist[src] = 0;
  queue[tail++] = src;
  while (head < tail) {
    int u = queue[head++];
    for (int e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
      int v = col_idx[e];
      if (dist[v] < 0) {
        dist[v] = dist[u] + 1;
        queue[tail++] = v;
      }
    }
  }
}

/* Dijkstra from src with non-negative edge lengths len[e] (one per CSR entry).
 * dist[v] = shortest-path length, INFINITY if unreachable.  Uses an O(n^2)
 * selection of the nearest unsettled vertex: slow and plain. */
void orc_dijkstra(int n, const int *row_ptr, const int *col_idx,
                  const double *len, int src, double *dist, char *done) {
  for (int v = 0; v < n; ++v) {
    dist[v] = INFINITY;
    done[v] = 0;
  }
  dist[src] = 0.0;
  for (int it = 0; it < n; ++it) {
    int u = -1;
    double best = INFINITY;
    for (int v = 0; v < n; ++v)
      if (!done[v] && dist[v] < best) {
        best = dist[v];
        u = v;
      }
    if (u < 0) break;
    done[u] = 1;
    for (int e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
      int v = col_idx[e];
      double cand = dist[u] + len[e];
      if (cand < dist[v]) dist[v] = cand;
    }
  }
}

/* All-pairs ideal distances into D[n][n] (diagonal 0).
 * len == NULL: unit edges (hop counts, BFS); otherwise Dijkstra.
 * Disconnected pairs: policy 0 returns ORC_ERR_DISCONNECTED; policy 1 sets
 * d_ij = (largest finite d over all pairs) + 1 -- the paper is silent on
 * disconnected graphs, this is the reading the library also takes. */
int orc_apsp(int n, const int *row_ptr, const int *col_idx, const double *len,
             int policy, double *D) {
  if (n < 0) return ORC_ERR_ARG;
  int *q = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  int *di = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  double *dd = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  char *done = (char *)malloc((size_t)(n > 0 ? n : 1));
  if (!q || !di || !dd || !done) {
    free(q); free(di); free(dd); free(done);
    return ORC_ERR_OOM;
  }
  int unreachable = 0;
  double dmax = 0.0;
  for (int s = 0; s < n; ++s) {
    if (len == NULL) {
      orc_bfs(n, row_ptr, col_idx, s, di, q);
      for (int v = 0; v < n; ++v) D[(size_t)s * n + v] = di[v] < 0 ? INFINITY : (double)di[v];
    } else {
      orc_dijkstra(n, row_ptr, col_idx, len, s, dd, done);
      for (int v = 0; v < n; ++v) D[(size_t)s * n + v] = dd[v];
    }
    for (int v = 0; v < n; ++v) {
      double x = D[(size_t)s * n + v];
      if (isinf(x)) unreachable = 1;
      else if (x > dmax) dmax = x;
    }
  }
  free(q); free(di); free(dd); free(done);
  if (unreachable) {
    if (policy != 1) return ORC_ERR_DISCONNECTED;
    for (size_t k = 0; k < (size_t)n * n; ++k)
      if (isinf(D[k])) D[k] = dmax + 1.0;
  }
  return ORC_OK;
}

/* Euclidean distance ||x_i - x_j|| in R^dim. */
static double orc_dist(int dim, const double *X, int i, int j) {
  double s = 0.0;
  for (int c = 0; c < dim; ++c) {
    double t = X[(size_t)i * dim + c] - X[(size_t)j * dim + c];
    s += t * t;
  }
  return sqrt(s);
}

/* Stress f(X) of Eq. (1) with w_ij = d_ij^{-2}: explicit loop over i < j. */
double orc_stress(int n, int dim, const double *X, const double *D) {
  double f = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      double d = D[(size_t)i * n + j];
      double w = 1.0 / (d * d);
      double e = orc_dist(dim, X, i, j) - d;
      f += w * e * e;
    }
  return f;
}

/* Majorization right-hand side b = L^Y Y at Y = X (Prop. 2.1 and Eq. (2-5)):
 * b_i = sum_{j != i} (-l^Y_ij)(x_i - x_j) = sum_{j!=i, x_j!=x_i} w_ij d_ij (x_i - x_j)/||x_i - x_j||.
 * (row sums of a Laplacian vanish, so (L^Y Y)_i = sum_j l_ij (y_j - y_i)). */
void orc_rhs(int n, int dim, const double *X, const double *D, double *b) {
  for (int i = 0; i < n; ++i) {
    for (int c = 0; c < dim; ++c) b[(size_t)i * dim + c] = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      double r = orc_dist(dim, X, i, j);
      if (r == 0.0) continue; /* l^Y_ij = 0 when y_i = y_j */
      double d = D[(size_t)i * n + j];
      double w = 1.0 / (d * d);
      double coef = w * d / r;
      for (int c = 0; c < dim; ++c)
        b[(size_t)i * dim + c] += coef * (X[(size_t)i * dim + c] - X[(size_t)j * dim + c]);
    }
  }
}

/* y = L^W P (Prop. 2.1): y_i = sum_{j != i} w_ij (p_i - p_j). */
void orc_lw_matvec(int n, int dim, const double *P, const double *D, double *y) {
  for (int i = 0; i < n; ++i) {
    for (int c = 0; c < dim; ++c) y[(size_t)i * dim + c] = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      double d = D[(size_t)i * n + j];
      double w = 1.0 / (d * d);
      for (int c = 0; c < dim; ++c)
        y[(size_t)i * dim + c] += w * (P[(size_t)i * dim + c] - P[(size_t)j * dim + c]);
    }
  }
}

/* Force F = (L^X - L^W) X = -(1/2) grad f(X):
 * F_i = sum_{j != i} w_ij (d_ij/||x_i - x_j|| - 1)(x_i - x_j); a coincident
 * pair contributes only its L^W part, which is zero there. */
void orc_forces(int n, int dim, const double *X, const double *D, double *F) {
  for (int i = 0; i < n; ++i) {
    for (int c = 0; c < dim; ++c) F[(size_t)i * dim + c] = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      double r = orc_dist(dim, X, i, j);
      double d = D[(size_t)i * n + j];
      double w = 1.0 / (d * d);
      double coef = (r == 0.0) ? -w : w * (d / r - 1.0);
      for (int c = 0; c < dim; ++c)
        F[(size_t)i * dim + c] += coef * (X[(size_t)i * dim + c] - X[(size_t)j * dim + c]);
    }
  }
}

/* --- single-row forms, for sampled checks at sizes where D[n][n] is too big --- */

/* Row i of F given row i of D (drow[j] = d_ij). */
void orc_force_row(int n, int dim, const double *X, int i, const double *drow, double *Fi) {
  for (int c = 0; c < dim; ++c) Fi[c] = 0.0;
  for (int j = 0; j < n; ++j) {
    if (j == i) continue;
    double r = orc_dist(dim, X, i, j);
    double d = drow[j];
    double w = 1.0 / (d * d);
    double coef = (r == 0.0) ? -w : w * (d / r - 1.0);
    for (int c = 0; c < dim; ++c)
      Fi[c] += coef * (X[(size_t)i * dim + c] - X[(size_t)j * dim + c]);
  }
}

/* Magnitude of the terms of row i of F, per coordinate:
 * A_ic = sum_{j != i} |w_ij (d_ij/||x_i - x_j|| - 1)(x_ic - x_jc)| (coincident
 * pairs: |w_ij (x_ic - x_jc)| = 0).  |F_ic| <= A_ic, with equality when every
 * term of the row has one sign; it is the scale of the rounding error of any
 * summation of the row's terms, so tolerances on F_ic are stated against it. */
void orc_force_row_abs(int n, int dim, const double *X, int i, const double *drow, double *Ai) {
  for (int c = 0; c < dim; ++c) Ai[c] = 0.0;
  for (int j = 0; j < n; ++j) {
    if (j == i) continue;
    double r = orc_dist(dim, X, i, j);
    double d = drow[j];
    double w = 1.0 / (d * d);
    double coef = (r == 0.0) ? -w : w * (d / r - 1.0);
    for (int c = 0; c < dim; ++c)
      Ai[c] += fabs(coef * (X[(size_t)i * dim + c] - X[(size_t)j * dim + c]));
  }
}

/* Row i of b = L^X X given row i of D. */
void orc_rhs_row(int n, int dim, const double *X, int i, const double *drow, double *bi) {
  for (int c = 0; c < dim; ++c) bi[c] = 0.0;
  for (int j = 0; j < n; ++j) {
    if (j == i) continue;
    double r = orc_dist(dim, X, i, j);
    if (r == 0.0) continue;
    double d = drow[j];
    double coef = (1.0 / (d * d)) * d / r;
    for (int c = 0; c < dim; ++c)
      bi[c] += coef * (X[(size_t)i * dim + c] - X[(size_t)j * dim + c]);
  }
}

/* Stress of Eq. (1) without storing D: one BFS per source row (unit edges),
 * then the row's pairs j > i, for the rows i0 <= i < i1 (the whole stress is
 * the sum over all rows; a caller may split the rows between processes and
 * add the parts).  Disconnected pairs take dfill (the caller passes max
 * finite d + 1, or a negative value to report an error). */
double orc_stress_stream_rows(int n, int dim, const double *X, const int *row_ptr,
                              const int *col_idx, double dfill, int i0, int i1, int *status) {
  int *q = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  int *di = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  *status = ORC_OK;
  if (!q || !di) {
    free(q); free(di);
    *status = ORC_ERR_OOM;
    return NAN;
  }
  double f = 0.0;
  for (int i = i0; i < i1; ++i) {
    orc_bfs(n, row_ptr, col_idx, i, di, q);
    for (int j = i + 1; j < n; ++j) {
      double d;
      if (di[j] < 0) {
        if (dfill < 0) {
          *status = ORC_ERR_DISCONNECTED;
          free(q); free(di);
          return NAN;
        }
        d = dfill;
      } else {
        d = (double)di[j];
      }
      double w = 1.0 / (d * d);
      double e = orc_dist(dim, X, i, j) - d;
      f += w * e * e;
    }
  }
  free(q); free(di);
  return f;
}

/* Stress of Eq. (1) of nl layouts of the same graph (layout l: dims[l]
 * coordinates, Xs[l] row-major), rows i0 <= i < i1, one BFS per row shared by
 * all layouts (the distances do not depend on the layout): f_out[l] receives
 * layout l's part. */
void orc_stress_stream_rows_multi(int n, int nl, const int *dims, const double *const *Xs,
                                  const int *row_ptr, const int *col_idx, double dfill, int i0,
                                  int i1, double *f_out, int *status) {
  int *q = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  int *di = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  *status = ORC_OK;
  for (int l = 0; l < nl; ++l) f_out[l] = 0.0;
  if (!q || !di) {
    free(q); free(di);
    *status = ORC_ERR_OOM;
    return;
  }
  for (int i = i0; i < i1; ++i) {
    orc_bfs(n, row_ptr, col_idx, i, di, q);
    for (int j = i + 1; j < n; ++j) {
      double d;
      if (di[j] < 0) {
        if (dfill < 0) {
          *status = ORC_ERR_DISCONNECTED;
          free(q); free(di);
          return;
        }
        d = dfill;
      } else {
        d = (double)di[j];
      }
      double w = 1.0 / (d * d);
      for (int l = 0; l < nl; ++l) {
        double e = orc_dist(dims[l], Xs[l], i, j) - d;
        f_out[l] += w * e * e;
      }
    }
  }
  free(q); free(di);
}

/* The whole stress of Eq. (1), streamed row by row (all rows). */
double orc_stress_stream(int n, int dim, const double *X, const int *row_ptr,
                         const int *col_idx, double dfill, int *status) {
  return orc_stress_stream_rows(n, dim, X, row_ptr, col_idx, dfill, 0, n, status);
}
