/* NVTX tool library for the trace tests (loaded by NVTX through
 * NVTX_INJECTION64_PATH).  It counts the ranges pushed in the "irk" domain by
 * name and by "parent>name", and records pops without a matching push.  The
 * test reads the counts back through the probe_* functions after loading the
 * same file with ctypes (one dlopen handle, one copy of the counters). */
#define NVTX_NO_IMPL
#include <nvtx3/nvToolsExt.h>
#include <pthread.h>
#include <stdio.h>
#include <string.h>

#define PROBE_KEYS 256
#define PROBE_DEPTH 64
#define PROBE_DOMAINS 16

struct probe_domain { char name[64]; };
static struct probe_domain domains[PROBE_DOMAINS];
static int ndomains;
static struct { char key[128]; int n; } counts[PROBE_KEYS];
static int nkeys, unmatched_pops, overflow, max_depth;
static pthread_mutex_t mu = PTHREAD_MUTEX_INITIALIZER;
static __thread const char* stack[PROBE_DEPTH];
static __thread int depth;

static void bump(const char* key) {
  for (int i = 0; i < nkeys; ++i)
    if (strcmp(counts[i].key, key) == 0) { counts[i].n += 1; return; }
  if (nkeys == PROBE_KEYS) { overflow += 1; return; }
  snprintf(counts[nkeys].key, sizeof counts[nkeys].key, "%s", key);
  counts[nkeys++].n = 1;
}

static int traced(nvtxDomainHandle_t d) {
  const struct probe_domain* p = (const struct probe_domain*)d;
  return p >= domains && p < domains + ndomains && strcmp(p->name, "irk") == 0;
}

static nvtxDomainHandle_t probe_create(const char* name) {
  pthread_mutex_lock(&mu);
  int i = ndomains < PROBE_DOMAINS ? ndomains++ : PROBE_DOMAINS - 1;
  snprintf(domains[i].name, sizeof domains[i].name, "%s", name ? name : "");
  pthread_mutex_unlock(&mu);
  return (nvtxDomainHandle_t)&domains[i];
}

static int probe_push(nvtxDomainHandle_t d, const nvtxEventAttributes_t* a) {
  if (!traced(d)) return 0;
  const char* name = (a && a->messageType == NVTX_MESSAGE_TYPE_ASCII) ? a->message.ascii : "?";
  char key[128];
  pthread_mutex_lock(&mu);
  bump(name);
  snprintf(key, sizeof key, "%s>%s", depth > 0 ? stack[depth - 1] : "", name);
  bump(key);
  if (depth < PROBE_DEPTH) stack[depth] = name; else overflow += 1;
  depth += 1;
  if (depth > max_depth) max_depth = depth;
  pthread_mutex_unlock(&mu);
  return depth - 1;
}

static int probe_pop(nvtxDomainHandle_t d) {
  if (!traced(d)) return 0;
  pthread_mutex_lock(&mu);
  if (depth == 0) unmatched_pops += 1; else depth -= 1;
  pthread_mutex_unlock(&mu);
  return depth;
}

int InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get_table) {
  const NvtxExportTableCallbacks* cb = (const NvtxExportTableCallbacks*)get_table(NVTX_ETID_CALLBACKS);
  NvtxFunctionTable table = 0;
  unsigned int size = 0;
  if (!cb || !cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE2, &table, &size)) return 0;
  if (size <= NVTX_CBID_CORE2_DomainCreateA) return 0;
  *table[NVTX_CBID_CORE2_DomainCreateA] = (NvtxFunctionPointer)probe_create;
  *table[NVTX_CBID_CORE2_DomainRangePushEx] = (NvtxFunctionPointer)probe_push;
  *table[NVTX_CBID_CORE2_DomainRangePop] = (NvtxFunctionPointer)probe_pop;
  return 1;
}

int probe_count(const char* key) {
  int n = 0;
  pthread_mutex_lock(&mu);
  for (int i = 0; i < nkeys; ++i)
    if (strcmp(counts[i].key, key) == 0) n = counts[i].n;
  pthread_mutex_unlock(&mu);
  return n;
}

int probe_errors(void) { return unmatched_pops + overflow; }
int probe_depth(void) { return depth; }
int probe_max_depth(void) { return max_depth; }
