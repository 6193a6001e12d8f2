/* Stand-in for libnvidia-ml.so.1 used by the CPU tests of the telemetry
 * sampler: the NVML query entry points the sampler resolves, returning
 * deterministic values, plus call counters the test reads back.  A setter is
 * exported too, so the test can check that the sampler never calls one.
 * FAKE_NVML_FAIL_INIT=1 makes nvmlInit_v2 fail; only device 0 exists. */
#include <stdatomic.h>
#include <stdlib.h>
#include <string.h>

typedef int nvmlReturn_t;
typedef void* nvmlDevice_t;
typedef struct { unsigned int gpu, memory; } nvmlUtilization_t;
typedef struct { unsigned long long total, free, used; } nvmlMemory_t;

static atomic_int n_init, n_shutdown, n_util, n_set;
static int dev0;

nvmlReturn_t nvmlInit_v2(void) {
  atomic_fetch_add(&n_init, 1);
  const char* f = getenv("FAKE_NVML_FAIL_INIT");
  return (f && *f == '1') ? 999 : 0;
}
nvmlReturn_t nvmlShutdown(void) { atomic_fetch_add(&n_shutdown, 1); return 0; }
nvmlReturn_t nvmlDeviceGetHandleByIndex_v2(unsigned int i, nvmlDevice_t* d) {
  if (i != 0) return 2; /* NVML_ERROR_INVALID_ARGUMENT */
  *d = &dev0;
  return 0;
}
nvmlReturn_t nvmlDeviceGetUtilizationRates(nvmlDevice_t d, nvmlUtilization_t* u) {
  int k = atomic_fetch_add(&n_util, 1);
  u->gpu = (unsigned)(k % 101);
  u->memory = 37;
  return d == &dev0 ? 0 : 2;
}
nvmlReturn_t nvmlDeviceGetMemoryInfo(nvmlDevice_t d, nvmlMemory_t* m) {
  m->total = 288ull << 30; m->used = 3ull << 30; m->free = m->total - m->used;
  return d == &dev0 ? 0 : 2;
}
nvmlReturn_t nvmlDeviceGetTemperature(nvmlDevice_t d, int sensor, unsigned int* t) {
  *t = sensor == 0 ? 41u : 0u;
  return d == &dev0 ? 0 : 2;
}
nvmlReturn_t nvmlDeviceGetPowerUsage(nvmlDevice_t d, unsigned int* mw) { (void)d; return 3; }
nvmlReturn_t nvmlDeviceGetClockInfo(nvmlDevice_t d, int type, unsigned int* mhz) {
  *mhz = type == 1 ? 2032u : 0u; /* NVML_CLOCK_SM = 1 */
  return d == &dev0 ? 0 : 2;
}
nvmlReturn_t nvmlDeviceSetApplicationsClocks(nvmlDevice_t d, unsigned a, unsigned b) {
  (void)d; (void)a; (void)b;
  atomic_fetch_add(&n_set, 1);
  return 0;
}

int fake_nvml_calls(const char* what) {
  if (!strcmp(what, "init")) return atomic_load(&n_init);
  if (!strcmp(what, "shutdown")) return atomic_load(&n_shutdown);
  if (!strcmp(what, "util")) return atomic_load(&n_util);
  if (!strcmp(what, "set")) return atomic_load(&n_set);
  return -1;
}
