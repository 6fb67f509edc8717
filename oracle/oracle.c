/*
 * CPU oracle for the worklist ForAll traversals -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * call this file. The CUDA path never links, loads or calls it, and it shares
 * no code with the CUDA path: it reads plain CSR arrays and writes plain
 * uint32 result arrays.
 *
 * Each function computes the unique fixed point that the data-driven kernel
 * must reach, by its plain textbook definition, serially:
 *
 *   oracle_bfs  -- level[v] = fewest edges on a directed path from a source to
 *                  v; INF = 0xFFFFFFFF when unreachable. This is the fixed point
 *                  of the level-by-level worklist BFS kernel of Sec. 4.1
 *                  (Listing "Level-by-level BFS kernel using a worklist"):
 *                  a source has level 0 and a vertex first reached in
 *                  invocation k (counting from 0) gets level k+1.
 *                  Method: FIFO queue (Moore/textbook BFS).
 *   oracle_sssp -- dist[v] = minimum over directed source->v paths of the sum of
 *                  the edge weights (int32 >= 0); INF when unreachable; with
 *                  several sources, the minimum over sources. Dijkstra with a
 *                  binary heap and lazy deletion, sums in uint64.
 *   oracle_cc   -- label[v] = smallest vertex id in v's connected component,
 *                  edges taken as undirected. Union-find (union by rank, path
 *                  halving), then the minimum id per root.
 *   oracle_msf  -- minimum spanning forest (Sec. 3.3's Boruvka example computes
 *                  it): the undirected edges {u, v} (u != v) of the CSR entries,
 *                  ordered by the key (w, min(u,v), max(u,v)), which makes the
 *                  forest unique (equal keys are copies of one edge). Kruskal:
 *                  sort the keys, keep each edge that joins two union-find sets.
 *
 * Return values: 0 on success; -1 invalid argument (vertex id out of range,
 * negative weight); -2 out of memory; -3 a distance does not fit below INF;
 * -4 more forest edges than n - 1 (cannot happen for a forest).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_INF 0xFFFFFFFFu

int oracle_bfs(uint32_t n, const uint32_t* row_ptr, const uint32_t* col, uint32_t nsrc,
               const uint32_t* src, uint32_t* level) {
  uint32_t i, head = 0, tail = 0;
  uint32_t* queue;
  for (i = 0; i < n; ++i) level[i] = ORACLE_INF;
  if (n == 0) return 0;
  queue = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n);
  if (!queue) return -2;
  for (i = 0; i < nsrc; ++i) {
    if (src[i] >= n) { free(queue); return -1; }
    if (level[src[i]] != 0) {
      level[src[i]] = 0;
      queue[tail++] = src[i];
    }
  }
  while (head < tail) {
    uint32_t u = queue[head++];
    uint32_t e;
    for (e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
      uint32_t v = col[e];
      if (v >= n) { free(queue); return -1; }
      if (level[v] == ORACLE_INF) {
        level[v] = level[u] + 1;
        queue[tail++] = v;
      }
    }
  }
  free(queue);
  return 0;
}

/* Binary min-heap of (key, vertex) pairs, lazy deletion. */
typedef struct {
  uint64_t key;
  uint32_t v;
} heap_item;

static void heap_push(heap_item* h, size_t* size, uint64_t key, uint32_t v) {
  size_t i = (*size)++;
  while (i > 0) {
    size_t p = (i - 1) / 2;
    if (h[p].key <= key) break;
    h[i] = h[p];
    i = p;
  }
  h[i].key = key;
  h[i].v = v;
}

static heap_item heap_pop(heap_item* h, size_t* size) {
  heap_item top = h[0];
  heap_item last = h[--(*size)];
  size_t i = 0, n = *size;
  for (;;) {
    size_t l = 2 * i + 1, r = l + 1, s = i;
    uint64_t sk = last.key;
    if (l < n && h[l].key < sk) { s = l; sk = h[l].key; }
    if (r < n && h[r].key < sk) { s = r; }
    if (s == i) break;
    h[i] = h[s];
    i = s;
  }
  if (n > 0) h[i] = last;
  return top;
}

int oracle_sssp(uint32_t n, const uint32_t* row_ptr, const uint32_t* col, const int32_t* w,
                uint32_t nsrc, const uint32_t* src, uint32_t* dist) {
  uint64_t* d;
  uint8_t* done;
  heap_item* heap;
  size_t hsize = 0, hcap;
  uint32_t i;
  int rc = 0;
  uint64_t m = n ? row_ptr[n] : 0;
  for (i = 0; i < n; ++i) dist[i] = ORACLE_INF;
  if (n == 0) return 0;
  d = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
  done = (uint8_t*)calloc(n, 1);
  hcap = (size_t)m + nsrc + 1;
  heap = (heap_item*)malloc(sizeof(heap_item) * hcap);
  if (!d || !done || !heap) { free(d); free(done); free(heap); return -2; }
  for (i = 0; i < n; ++i) d[i] = UINT64_MAX;
  for (i = 0; i < nsrc; ++i) {
    if (src[i] >= n) { rc = -1; goto out; }
    if (d[src[i]] != 0) {
      d[src[i]] = 0;
      heap_push(heap, &hsize, 0, src[i]);
    }
  }
  while (hsize > 0) {
    heap_item it = heap_pop(heap, &hsize);
    uint32_t u = it.v, e;
    if (done[u] || it.key != d[u]) continue;
    done[u] = 1;
    for (e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
      uint32_t v = col[e];
      uint64_t nd;
      if (v >= n || w[e] < 0) { rc = -1; goto out; }
      nd = d[u] + (uint64_t)w[e];
      if (nd < d[v]) {
        d[v] = nd;
        heap_push(heap, &hsize, nd, v);
      }
    }
  }
  for (i = 0; i < n; ++i) {
    if (d[i] == UINT64_MAX) continue;
    if (d[i] >= ORACLE_INF) { rc = -3; goto out; }
    dist[i] = (uint32_t)d[i];
  }
out:
  free(d);
  free(done);
  free(heap);
  return rc;
}

static uint32_t uf_find(uint32_t* parent, uint32_t x) {
  while (parent[x] != x) {
    parent[x] = parent[parent[x]]; /* path halving */
    x = parent[x];
  }
  return x;
}

int oracle_cc(uint32_t n, const uint32_t* row_ptr, const uint32_t* col, uint32_t* label) {
  uint32_t* parent;
  uint8_t* rank;
  uint32_t* minid;
  uint32_t u, e;
  if (n == 0) return 0;
  parent = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n);
  rank = (uint8_t*)calloc(n, 1);
  minid = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n);
  if (!parent || !rank || !minid) { free(parent); free(rank); free(minid); return -2; }
  for (u = 0; u < n; ++u) parent[u] = u;
  for (u = 0; u < n; ++u) {
    for (e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
      uint32_t v = col[e], a, b;
      if (v >= n) { free(parent); free(rank); free(minid); return -1; }
      a = uf_find(parent, u);
      b = uf_find(parent, v);
      if (a == b) continue;
      if (rank[a] < rank[b]) { uint32_t t = a; a = b; b = t; }
      parent[b] = a; /* union by rank */
      if (rank[a] == rank[b]) rank[a]++;
    }
  }
  for (u = 0; u < n; ++u) minid[u] = ORACLE_INF;
  for (u = 0; u < n; ++u) {
    uint32_t r = uf_find(parent, u);
    if (u < minid[r]) minid[r] = u;
  }
  for (u = 0; u < n; ++u) label[u] = minid[uf_find(parent, u)];
  free(parent);
  free(rank);
  free(minid);
  return 0;
}

/* ---------------------------------------------------------------- minimum spanning forest */

typedef struct {
  int32_t w;
  uint32_t u, v; /* u < v */
} msf_edge;

static int msf_key_cmp(const void* pa, const void* pb) {
  const msf_edge* a = (const msf_edge*)pa;
  const msf_edge* b = (const msf_edge*)pb;
  if (a->w != b->w) return a->w < b->w ? -1 : 1;
  if (a->u != b->u) return a->u < b->u ? -1 : 1;
  if (a->v != b->v) return a->v < b->v ? -1 : 1;
  return 0;
}

/* Kruskal's algorithm over the key order (w, min(u,v), max(u,v)). Writes the
 * kept edges in key order (out_u < out_v; capacity n - 1 each), their number
 * and the sum of their weights. */
int oracle_msf(uint32_t n, const uint32_t* row_ptr, const uint32_t* col, const int32_t* w, uint32_t* out_u,
               uint32_t* out_v, int32_t* out_w, uint32_t* count, uint64_t* total) {
  uint64_t m = n ? row_ptr[n] : 0, k = 0, e;
  uint32_t u, kept = 0;
  uint64_t sum = 0;
  msf_edge* edges;
  uint32_t* parent;
  *count = 0;
  *total = 0;
  if (n == 0) return 0;
  edges = (msf_edge*)malloc(sizeof(msf_edge) * (size_t)(m ? m : 1));
  parent = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n);
  if (!edges || !parent) {
    free(edges);
    free(parent);
    return -2;
  }
  for (u = 0; u < n; ++u) {
    parent[u] = u;
    for (e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
      uint32_t v = col[e];
      if (v >= n || w[e] < 0) {
        free(edges);
        free(parent);
        return -1;
      }
      if (v == u) continue; /* a self-loop joins nothing */
      edges[k].w = w[e];
      edges[k].u = u < v ? u : v;
      edges[k].v = u < v ? v : u;
      ++k;
    }
  }
  qsort(edges, (size_t)k, sizeof(msf_edge), msf_key_cmp);
  for (e = 0; e < k; ++e) {
    uint32_t a = uf_find(parent, edges[e].u), b = uf_find(parent, edges[e].v);
    if (a == b) continue; /* closes a cycle: every cycle edge before it is lighter */
    if (kept + 1 >= n) { /* a forest on n vertices has at most n - 1 edges */
      free(edges);
      free(parent);
      return -4;
    }
    parent[a > b ? a : b] = a < b ? a : b;
    out_u[kept] = edges[e].u;
    out_v[kept] = edges[e].v;
    out_w[kept] = edges[e].w;
    sum += (uint64_t)edges[e].w;
    ++kept;
  }
  *count = kept;
  *total = sum;
  free(edges);
  free(parent);
  return 0;
}
