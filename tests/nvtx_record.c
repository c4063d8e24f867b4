/* NVTX injection library used by tests/test_gpu_nvtx.py: NVTX loads it from
 * NVTX_INJECTION64_PATH at the first NVTX call and calls
 * InitializeInjectionNvtx2, which installs two handlers in the core callback
 * module (the public interface of nvtx3/nvtxDetail/nvtxTypes.h).  Every
 * nvtxRangePushA message and every nvtxRangePop is written, one per line, to
 * the file named by COLDEN_NVTX_LOG. */
#include <stdio.h>
#include <stdlib.h>

#include <nvtx3/nvToolsExt.h>

static FILE *g_log;

static int record_push(const char *message)
{
    if (g_log) fprintf(g_log, "push %s\n", message ? message : "");
    return 0;
}

static int record_pop(void)
{
    if (g_log) fprintf(g_log, "pop\n");
    return 0;
}

static void close_log(void)
{
    if (g_log) fclose(g_log);
}

int InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get)
{
    const NvtxExportTableCallbacks *cb = (const NvtxExportTableCallbacks *)get(NVTX_ETID_CALLBACKS);
    NvtxFunctionTable table = 0;
    unsigned int n = 0;
    const char *path = getenv("COLDEN_NVTX_LOG");
    if (!cb || !path || !cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE, &table, &n) || n <= NVTX_CBID_CORE_RangePop)
        return 0;
    g_log = fopen(path, "w");
    if (!g_log) return 0;
    atexit(close_log);
    *table[NVTX_CBID_CORE_RangePushA] = (NvtxFunctionPointer)record_push;
    *table[NVTX_CBID_CORE_RangePop] = (NvtxFunctionPointer)record_pop;
    return 1;
}
