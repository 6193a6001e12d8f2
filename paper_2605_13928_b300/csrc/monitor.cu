// monitor.cu -- GPU telemetry sampler with the four verbs of the paper's
// CudaMon package (Sec. 2: start a sampler with a period and a device index,
// add named timestamps, stop it, parse the collected trace).  Host code only.
//
// A background thread queries NVML every `period` seconds for GPU and memory
// utilisation, memory in use, temperature, power draw and SM clock, and keeps
// the rows (and, if asked, appends them to a CSV file).  Every query is
// read-only: nothing changes any setting of the device.  NVML is loaded at run
// time (libnvidia-ml.so.1, or the library named by $TSNE_NVML_LIB), so the
// sampler works wherever the NVIDIA driver is present and fails cleanly elsewhere.
#include <dlfcn.h>
#include <nvml.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"

namespace {

struct NvmlApi {
  void* handle = nullptr;
  nvmlReturn_t (*init)() = nullptr;
  nvmlReturn_t (*shutdown)() = nullptr;
  nvmlReturn_t (*by_index)(unsigned, nvmlDevice_t*) = nullptr;
  nvmlReturn_t (*util)(nvmlDevice_t, nvmlUtilization_t*) = nullptr;
  nvmlReturn_t (*mem)(nvmlDevice_t, nvmlMemory_t*) = nullptr;
  nvmlReturn_t (*temp)(nvmlDevice_t, nvmlTemperatureSensors_t, unsigned*) = nullptr;
  nvmlReturn_t (*power)(nvmlDevice_t, unsigned*) = nullptr;
  nvmlReturn_t (*clock)(nvmlDevice_t, nvmlClockType_t, unsigned*) = nullptr;

  bool load() {
    const char* path = getenv("TSNE_NVML_LIB");
    handle = dlopen(path && *path ? path : "libnvidia-ml.so.1", RTLD_NOW | RTLD_LOCAL);
    if (!handle) return false;
    init = reinterpret_cast<nvmlReturn_t (*)()>(dlsym(handle, "nvmlInit_v2"));
    shutdown = reinterpret_cast<nvmlReturn_t (*)()>(dlsym(handle, "nvmlShutdown"));
    by_index = reinterpret_cast<nvmlReturn_t (*)(unsigned, nvmlDevice_t*)>(
        dlsym(handle, "nvmlDeviceGetHandleByIndex_v2"));
    util = reinterpret_cast<nvmlReturn_t (*)(nvmlDevice_t, nvmlUtilization_t*)>(
        dlsym(handle, "nvmlDeviceGetUtilizationRates"));
    mem = reinterpret_cast<nvmlReturn_t (*)(nvmlDevice_t, nvmlMemory_t*)>(
        dlsym(handle, "nvmlDeviceGetMemoryInfo"));
    temp = reinterpret_cast<nvmlReturn_t (*)(nvmlDevice_t, nvmlTemperatureSensors_t, unsigned*)>(
        dlsym(handle, "nvmlDeviceGetTemperature"));
    power = reinterpret_cast<nvmlReturn_t (*)(nvmlDevice_t, unsigned*)>(
        dlsym(handle, "nvmlDeviceGetPowerUsage"));
    clock = reinterpret_cast<nvmlReturn_t (*)(nvmlDevice_t, nvmlClockType_t, unsigned*)>(
        dlsym(handle, "nvmlDeviceGetClockInfo"));
    return init && shutdown && by_index && util && mem && temp && power && clock;
  }
};

struct Row {
  double t, gpu_util, mem_util, mem_used_mb, temp_c, power_w, sm_mhz;
};

struct Event {
  double t;
  std::string name;
};

}  // namespace

struct tsne_mon {
  NvmlApi api;
  nvmlDevice_t dev{};
  double period = 1.0;
  std::chrono::steady_clock::time_point t0;
  FILE* csv = nullptr;
  std::vector<Row> rows;
  std::vector<Event> events;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  bool stopped = false;
  std::thread th;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }

  void sample() {
    Row r{};
    r.t = now();
    nvmlUtilization_t u{};
    nvmlMemory_t m{};
    unsigned tc = 0, mw = 0, mhz = 0;
    r.gpu_util = api.util(dev, &u) == NVML_SUCCESS ? u.gpu : -1.0;
    r.mem_util = r.gpu_util >= 0 ? u.memory : -1.0;
    r.mem_used_mb = api.mem(dev, &m) == NVML_SUCCESS ? (double)m.used / (1024.0 * 1024.0) : -1.0;
    r.temp_c = api.temp(dev, NVML_TEMPERATURE_GPU, &tc) == NVML_SUCCESS ? tc : -1.0;
    r.power_w = api.power(dev, &mw) == NVML_SUCCESS ? mw / 1000.0 : -1.0;
    r.sm_mhz = api.clock(dev, NVML_CLOCK_SM, &mhz) == NVML_SUCCESS ? mhz : -1.0;
    std::lock_guard<std::mutex> lk(mu);
    rows.push_back(r);
    if (csv) {
      fprintf(csv, "sample,%.6f,%.1f,%.1f,%.1f,%.1f,%.3f,%.0f,\n", r.t, r.gpu_util, r.mem_util,
              r.mem_used_mb, r.temp_c, r.power_w, r.sm_mhz);
    }
  }

  void loop() {
    std::unique_lock<std::mutex> lk(mu);
    auto next = std::chrono::steady_clock::now();
    while (!stop) {
      lk.unlock();
      sample();
      lk.lock();
      next += std::chrono::duration_cast<std::chrono::steady_clock::duration>(
          std::chrono::duration<double>(period));
      cv.wait_until(lk, next, [this] { return stop; });
    }
  }
};

extern "C" {

tsne_mon* tsne_mon_start(int device_index, double period_s, const char* csv_path, int* err) {
  auto fail = [err](int code) -> tsne_mon* {
    if (err) *err = code;
    return nullptr;
  };
  if (device_index < 0 || !(period_s >= 0.001)) return fail(TSNE_ERR_ARG);
  tsne_mon* m = new tsne_mon();
  if (!m->api.load()) {
    if (m->api.handle) dlclose(m->api.handle);
    delete m;
    return fail(TSNE_ERR_DEVICE);
  }
  if (m->api.init() != NVML_SUCCESS) {
    dlclose(m->api.handle);
    delete m;
    return fail(TSNE_ERR_DEVICE);
  }
  if (m->api.by_index((unsigned)device_index, &m->dev) != NVML_SUCCESS) {
    m->api.shutdown();
    dlclose(m->api.handle);
    delete m;
    return fail(TSNE_ERR_ARG);
  }
  if (csv_path && *csv_path) {
    m->csv = fopen(csv_path, "w");
    if (!m->csv) {
      m->api.shutdown();
      dlclose(m->api.handle);
      delete m;
      return fail(TSNE_ERR_ARG);
    }
    fprintf(m->csv, "kind,t_s,gpu_util_pct,mem_util_pct,mem_used_mb,temp_c,power_w,sm_mhz,event\n");
  }
  m->period = period_s;
  m->t0 = std::chrono::steady_clock::now();
  m->th = std::thread([m] { m->loop(); });
  if (err) *err = TSNE_OK;
  return m;
}

int tsne_mon_mark(tsne_mon* m, const char* name) {
  if (!m || !name) return TSNE_ERR_ARG;
  std::lock_guard<std::mutex> lk(m->mu);
  if (m->stopped) return TSNE_ERR_ARG;
  const double t = m->now();
  m->events.push_back(Event{t, std::string(name)});
  if (m->csv) fprintf(m->csv, "event,%.6f,,,,,,,%s\n", t, name);
  return TSNE_OK;
}

int tsne_mon_stop(tsne_mon* m) {
  if (!m) return TSNE_ERR_ARG;
  {
    std::lock_guard<std::mutex> lk(m->mu);
    if (m->stopped) return TSNE_OK;
    m->stop = true;
  }
  m->cv.notify_all();
  if (m->th.joinable()) m->th.join();
  std::lock_guard<std::mutex> lk(m->mu);
  m->stopped = true;
  if (m->csv) {
    fclose(m->csv);
    m->csv = nullptr;
  }
  m->api.shutdown();
  return TSNE_OK;
}

int64_t tsne_mon_count(tsne_mon* m, int what) {
  if (!m) return TSNE_ERR_ARG;
  std::lock_guard<std::mutex> lk(m->mu);
  return what == 0 ? (int64_t)m->rows.size() : (int64_t)m->events.size();
}

int tsne_mon_samples(tsne_mon* m, double* out, int64_t cap_rows) {
  if (!m || !out || cap_rows < 0) return TSNE_ERR_ARG;
  std::lock_guard<std::mutex> lk(m->mu);
  const int64_t k = (int64_t)m->rows.size() < cap_rows ? (int64_t)m->rows.size() : cap_rows;
  for (int64_t i = 0; i < k; i++) {
    const Row& r = m->rows[i];
    const double v[7] = {r.t, r.gpu_util, r.mem_util, r.mem_used_mb, r.temp_c, r.power_w, r.sm_mhz};
    memcpy(out + 7 * i, v, sizeof(v));
  }
  return TSNE_OK;
}

int tsne_mon_event(tsne_mon* m, int64_t i, double* t, char* name, int cap) {
  if (!m || !t || !name || cap < 1) return TSNE_ERR_ARG;
  std::lock_guard<std::mutex> lk(m->mu);
  if (i < 0 || i >= (int64_t)m->events.size()) return TSNE_ERR_ARG;
  *t = m->events[i].t;
  snprintf(name, (size_t)cap, "%s", m->events[i].name.c_str());
  return TSNE_OK;
}

void tsne_mon_free(tsne_mon* m) {
  if (!m) return;
  tsne_mon_stop(m);
  if (m->api.handle) dlclose(m->api.handle);
  delete m;
}

}  // extern "C"
