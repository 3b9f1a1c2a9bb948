/*
 * A minimal NVTX tool for the tests: loaded by NVTX through
 * NVTX_INJECTION64_PATH, it writes every range push ("+name") and pop ("-")
 * of the process to the file named by AWPM_NVTX_LOG.
 */
#include <stdio.h>
#include <stdlib.h>

#include <nvtx3/nvToolsExt.h>

static FILE *g_log;

static int log_push(const char *msg)
{
    if (g_log) {
        fprintf(g_log, "+%s\n", msg ? msg : "");
        fflush(g_log);
    }
    return 0;
}

static int log_pop(void)
{
    if (g_log) {
        fputs("-\n", g_log);
        fflush(g_log);
    }
    return 0;
}

int InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get_table)
{
    const NvtxExportTableCallbacks *cb =
        (const NvtxExportTableCallbacks *)get_table(NVTX_ETID_CALLBACKS);
    NvtxFunctionTable table = 0;
    unsigned int size = 0;
    if (!cb || !cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE, &table, &size) ||
        size <= NVTX_CBID_CORE_RangePop)
        return 0;
    *table[NVTX_CBID_CORE_RangePushA] = (NvtxFunctionPointer)log_push;
    *table[NVTX_CBID_CORE_RangePop] = (NvtxFunctionPointer)log_pop;
    const char *path = getenv("AWPM_NVTX_LOG");
    g_log = path ? fopen(path, "w") : NULL;
    return 1;
}
