/* nvtx_record.c -- a minimal NVTX injection library for the tests: it
 * records every range push (the range's message) and pop, one line each,
 * to the file named by AF_NVTX_LOG.  Loaded by the NVTX header code of the
 * library under test when NVTX_INJECTION64_PATH names this file; it uses
 * only the callback interface that nvtx3's headers declare. */
#include <stdio.h>
#include <stdlib.h>

#include <nvtx3/nvToolsExt.h>

static FILE *out;

static int rec_push(const char *msg) {
  if (out) {
    fprintf(out, "push %s\n", msg ? msg : "");
    fflush(out);
  }
  return 0;
}

static int rec_pop(void) {
  if (out) {
    fprintf(out, "pop\n");
    fflush(out);
  }
  return 0;
}

int InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get_table) {
  const char *path = getenv("AF_NVTX_LOG");
  out = path ? fopen(path, "w") : NULL;
  const NvtxExportTableCallbacks *cb = (const NvtxExportTableCallbacks *)get_table(NVTX_ETID_CALLBACKS);
  if (!cb || !out) return 0;
  NvtxFunctionTable table = 0;
  unsigned int size = 0;
  if (!cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE, &table, &size) || !table) return 0;
  if (size >= NVTX_CBID_CORE_RangePushA) *table[NVTX_CBID_CORE_RangePushA] = (NvtxFunctionPointer)rec_push;
  if (size >= NVTX_CBID_CORE_RangePop) *table[NVTX_CBID_CORE_RangePop] = (NvtxFunctionPointer)rec_pop;
  return 1;
}
