// Event-based per-kernel timing (sem_profile_begin / sem_profile_end).
#include <cstring>
#include <string>
#include <vector>

#include "sem_internal.h"

namespace sem {
namespace {
struct Rec {
  int kid;
  cudaEvent_t a, b;
};
bool g_on = false;
std::vector<std::string> g_names;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
size_t g_used = 0;

cudaEvent_t take() {
  if (g_used == g_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    g_pool.push_back(e);
  }
  return g_pool[g_used++];
}
}  // namespace

int prof_begin_kernel(const char* name, cudaStream_t st) {
  if (!g_on || g_recs.size() >= (1u << 16)) return -1;
  int kid = -1;
  for (size_t k = 0; k < g_names.size(); ++k)
    if (g_names[k] == name) kid = (int)k;
  if (kid < 0) {
    if (g_names.size() >= SEM_PROFILE_MAX) return -1;
    g_names.push_back(name);
    kid = (int)g_names.size() - 1;
  }
  Rec r{kid, take(), take()};
  if (!r.a || !r.b) return -1;
  cudaEventRecord(r.a, st);
  g_recs.push_back(r);
  return (int)g_recs.size() - 1;
}

void prof_end_kernel(int rec, cudaStream_t st) {
  if (rec < 0) return;
  cudaEventRecord(g_recs[rec].b, st);
}

}  // namespace sem

using namespace sem;

extern "C" int sem_profile_begin(void) {
  g_on = true;
  g_names.clear();
  g_recs.clear();
  g_used = 0;
  return SEM_OK;
}

extern "C" int sem_profile_end(sem_profile_out* out) {
  if (!out) return fail(SEM_ERR_ARG, "NULL argument");
  std::memset(out, 0, sizeof(*out));
  g_on = false;
  for (auto& r : g_recs) {
    SEM_CUDA_TRY(cudaEventSynchronize(r.b));
    float ms = 0.f;
    SEM_CUDA_TRY(cudaEventElapsedTime(&ms, r.a, r.b));
    out->ms_total[r.kid] += ms;
    out->launches[r.kid] += 1;
  }
  out->n_kernels = (int)g_names.size();
  for (size_t k = 0; k < g_names.size(); ++k)
    std::strncpy(out->name[k], g_names[k].c_str(), sizeof(out->name[k]) - 1);
  g_recs.clear();
  g_used = 0;
  return SEM_OK;
}
