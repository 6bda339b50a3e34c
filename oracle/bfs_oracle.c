/*
 * Oracle: serial breadth-first search distances (plain C).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load or run this file.  The CUDA library
 * shares no code with it and never calls it.
 *
 * What it computes.  The paper (Section 1 and the start of Section 2) defines
 * BFS as exploring a graph level by level from a source; the distance of a
 * vertex is the level at which it is reached, i.e. the number of edges on a
 * shortest path from the source.  Listing 1 relaxes an edge (src, dst) when
 * dist[src] + 1 < dist[dst] with unvisited vertices holding MAX_DISTANCE, and
 * the bottom-up phase of Listings 2 and 3 gives an unvisited vertex distance
 * depth + 1 as soon as one neighbour lies in the current frontier.  Both reach
 * the same unique result: the shortest-path hop count.  The serial FIFO-queue
 * BFS (the "serial BFS" the paper uses as its baseline in Section 3) is that
 * definition written out, and it is what this file implements.
 *
 * Readings: unreachable vertices hold -1 (the paper's MAX_DISTANCE sentinel,
 * encoded as -1 in the library's int32 output).  The graph is a CSR with
 * int64 row pointers and int32 neighbour ids; for an undirected graph every
 * edge is stored in both directions.  Self-loops and repeated entries are
 * allowed and change nothing.
 *
 * Pins (tests, CPU only): brute-force repeated relaxation on every graph with
 * up to five vertices and on random graphs up to 64 vertices; closed forms for
 * paths, stars, complete graphs, cycles, 2-D grids and disjoint unions; and the
 * BFS invariants (d[src] = 0, |d(u) - d(v)| <= 1 on every edge, a parent at
 * d - 1 for every reached vertex, -1 exactly off the source's component as
 * found by union-find).
 */
#include <stdint.h>
#include <stdlib.h>

/*
 * dist[v] = number of edges on a shortest path from src to v, or -1.
 * row_ptr has n+1 entries, col has row_ptr[n] entries.
 * Returns 0, or -1 for bad arguments (n < 1, src outside [0, n), a neighbour
 * id outside [0, n)) or -2 when the queue cannot be allocated.
 */
int oracle_bfs(int64_t n, const int64_t *row_ptr, const int32_t *col, int64_t src, int32_t *dist) {
    if (n < 1 || src < 0 || src >= n) return -1;
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!queue) return -2;
    for (int64_t v = 0; v < n; ++v) dist[v] = -1;
    int64_t head = 0, tail = 0;
    dist[src] = 0;
    queue[tail++] = src;
    while (head < tail) {
        int64_t u = queue[head++];
        for (int64_t j = row_ptr[u]; j < row_ptr[u + 1]; ++j) {
            int64_t v = col[j];
            if (v < 0 || v >= n) {
                free(queue);
                return -1;
            }
            if (dist[v] == -1) {
                dist[v] = dist[u] + 1;
                queue[tail++] = v;
            }
        }
    }
    free(queue);
    return 0;
}
