/* NVTX injection library used by the tracing test (test infrastructure, not part of
 * the product).  Loaded through NVTX_INJECTION64_PATH, it takes the domain create,
 * push and pop slots of the NVTX core-2 module and appends one line per event to a
 * buffer that the test reads with nvtx_record_log(). */
#include <stdio.h>
#include <string.h>

#include <nvtx3/nvToolsExt.h>

#define MAX_DOMAINS 16
static char g_domains[MAX_DOMAINS][64];
static int g_ndomains;
static char g_log[1 << 16];
static size_t g_len;

static void append(const char *kind, nvtxDomainHandle_t d, const char *name)
{
    const long i = (long)(size_t)d - 1;
    const char *dn = (i >= 0 && i < g_ndomains) ? g_domains[i] : "?";
    const int n = snprintf(g_log + g_len, sizeof g_log - g_len, "%s %s %s\n", kind, dn, name ? name : "");
    if (n > 0 && g_len + (size_t)n < sizeof g_log) g_len += (size_t)n;
}

static nvtxDomainHandle_t NVTX_API rec_domain_create(const char *name)
{
    if (g_ndomains == MAX_DOMAINS) return (nvtxDomainHandle_t)0;
    snprintf(g_domains[g_ndomains], sizeof g_domains[0], "%s", name);
    ++g_ndomains;
    return (nvtxDomainHandle_t)(size_t)g_ndomains;      /* handle = index + 1 */
}

static int NVTX_API rec_push(nvtxDomainHandle_t d, const nvtxEventAttributes_t *a)
{
    const char *name = (a && a->messageType == NVTX_MESSAGE_TYPE_ASCII) ? a->message.ascii : "";
    if (a && a->payloadType == NVTX_PAYLOAD_TYPE_INT64) {      /* name#payload */
        char buf[96];
        snprintf(buf, sizeof buf, "%s#%lld", name, (long long)a->payload.llValue);
        append("push", d, buf);
    } else {
        append("push", d, name);
    }
    return 0;
}

static int NVTX_API rec_pop(nvtxDomainHandle_t d)
{
    append("pop", d, "");
    return 0;
}

const char *nvtx_record_log(void) { return g_log; }

int NVTX_API InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get_table)
{
    const NvtxExportTableCallbacks *cb = (const NvtxExportTableCallbacks *)get_table(NVTX_ETID_CALLBACKS);
    NvtxFunctionTable t = 0;
    unsigned int n = 0;
    if (!cb || !cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE2, &t, &n) || !t)
        return 0;
    if (n <= NVTX_CBID_CORE2_DomainCreateA) return 0;
    *t[NVTX_CBID_CORE2_DomainCreateA] = (NvtxFunctionPointer)rec_domain_create;
    *t[NVTX_CBID_CORE2_DomainRangePushEx] = (NvtxFunctionPointer)rec_push;
    *t[NVTX_CBID_CORE2_DomainRangePop] = (NvtxFunctionPointer)rec_pop;
    return 1;
}
