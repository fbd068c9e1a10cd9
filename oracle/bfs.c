/*
 * Breadth-first search distances -- oracle (test infrastructure only; never
 * linked into the CUDA library).
 *
 * The frontier-based BFS of the thesis (Sec. 4.3, the inner-array BFS
 * benchmark; run as a parallel_do per frontier level, ended by a reduce)
 * computes, for every vertex, the number of edges on a shortest path from
 * the start vertex.  Its plain definition is the breadth-first search below
 * (a FIFO queue over a CSR graph); unreachable vertices keep INT32_MAX.
 */
#include <stdlib.h>
#include "oracle.h"

int orc_bfs(int n, const int32_t* row_ptr, const int32_t* col, int source, int32_t* dist, int* levels) {
  if (n < 1 || !row_ptr || !col || !dist || source < 0 || source >= n) return -1;
  int* q = (int*)malloc(sizeof(int) * (size_t)n);
  for (int v = 0; v < n; ++v) dist[v] = INT32_MAX;
  int head = 0, tail = 0, maxd = 0;
  dist[source] = 0;
  q[tail++] = source;
  while (head < tail) {
    const int v = q[head++];
    for (int e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
      const int w = col[e];
      if (dist[w] == INT32_MAX) {
        dist[w] = dist[v] + 1;
        if (dist[w] > maxd) maxd = dist[w];
        q[tail++] = w;
      }
    }
  }
  if (levels) *levels = maxd + 1;
  free(q);
  return 0;
}
