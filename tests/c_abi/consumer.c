/* A plain C99 user of the library: includes only include/bfs.h, links
 * libbfs_gb300.so (or its bounds-checking twin) and makes calls that need no
 * GPU.  Exit status 0 when every answer is the documented one. */
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "bfs.h"

static int check(const char* what, int got, int want) {
  if (got != want) {
    fprintf(stderr, "%s: status %d, expected %d (%s)\n", what, got, want, bfs_last_error());
    return 1;
  }
  printf("%s: %d (%s)\n", what, got, bfs_last_error());
  return 0;
}

int main(int argc, char** argv) {
  int bad = 0;
  const int want_checked = argc > 1 && strcmp(argv[1], "--checked") == 0;
  int32_t buf[4] = {0, 0, 0, 0};
  int64_t off[3] = {0, 1, 2};
  int32_t adj[2] = {1, 0};
  bfs_graph* g = NULL;
  printf("version: %s\n", bfs_version());
  if (bfs_bounds_checked() != want_checked) {
    fprintf(stderr, "bfs_bounds_checked() = %d\n", bfs_bounds_checked());
    bad = 1;
  }
  bad |= check("bfs_run without a graph", bfs_run(NULL, 0, buf, buf, NULL, NULL), BFS_ERR_INVALID_ARG);
  bad |= check("bfs_graph_create with n = 0", bfs_graph_create(off, adj, 0, 2, BFS_HOST_PTRS, &g),
               BFS_ERR_INVALID_ARG);
  bad |= check("bfs_run_static with a source outside [0, n)",
               bfs_run_static(off, adj, 2, 2, 7, buf, buf, NULL), BFS_ERR_INVALID_ARG);
  {
    bfs_tile_info info;
    bad |= check("bfs_graph_tiles without a graph", bfs_graph_tiles(NULL, 0, 0, &info, NULL), BFS_ERR_INVALID_ARG);
  }
  {
    int32_t cnt = 0;
    bad |= check("bfs_spmsv_sorted without a graph", bfs_spmsv_sorted(NULL, buf, 1, NULL, buf, buf, &cnt, NULL),
                 BFS_ERR_INVALID_ARG);
    bad |= check("bfs_run_sorted without a graph", bfs_run_sorted(NULL, 0, buf, buf, NULL), BFS_ERR_INVALID_ARG);
  }
  {
    bfs_half_info hinfo;
    bad |= check("bfs_graph_half without a graph", bfs_graph_half(NULL, &hinfo, NULL), BFS_ERR_INVALID_ARG);
    bad |= check("bfs_run_half without a graph", bfs_run_half(NULL, 0, buf, buf, NULL), BFS_ERR_INVALID_ARG);
  }
  if (g != NULL) {
    fprintf(stderr, "a failed create left a graph behind\n");
    bad = 1;
  }
  return bad;
}
