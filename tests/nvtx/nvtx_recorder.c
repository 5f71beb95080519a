/* A minimal NVTX tool for tests: loaded through NVTX_INJECTION64_PATH, it
 * records every nvtxRangePushA / nvtxRangePop of the process, one line each,
 * in the file named by NVTX_RECORD_PATH.  The types mirror the NVTX 3 tool
 * interface (export table 1 = callbacks; module 1 = core; core callback 9 =
 * RangePushA, 11 = RangePop). */
#include <stddef.h>
#include <stdio.h>
#include <stdlib.h>

typedef void (*nvtx_fn)(void);
typedef nvtx_fn** nvtx_table;
typedef struct {
  size_t struct_size;
  int (*get_module_function_table)(int module, nvtx_table* out_table, unsigned int* out_size);
} nvtx_callbacks;
typedef const void* (*nvtx_get_export_table)(unsigned int id);

static FILE* record;

static int on_push(const char* message) {
  fprintf(record, "push %s\n", message);
  fflush(record);
  return 0;
}

static int on_pop(void) {
  fprintf(record, "pop\n");
  fflush(record);
  return 0;
}

int InitializeInjectionNvtx2(nvtx_get_export_table get_export_table) {
  const char* path = getenv("NVTX_RECORD_PATH");
  const nvtx_callbacks* cb = (const nvtx_callbacks*)get_export_table(1);
  nvtx_table core = NULL;
  unsigned int size = 0;
  if (!path || !cb || !cb->get_module_function_table(1, &core, &size) || size <= 11) return 0;
  record = fopen(path, "w");
  if (!record) return 0;
  *core[9] = (nvtx_fn)on_push;
  *core[11] = (nvtx_fn)on_pop;
  return 1;
}
