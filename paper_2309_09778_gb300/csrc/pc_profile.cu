// Per-stage event timing for the C ABI.  A fixed pool of event pairs is
// created on first enable; each launch inside a call takes the next pair.
#include <mutex>

#include "pc_kernels.cuh"
#include "pc_profile.cuh"

namespace pc {
namespace {
constexpr int kPool = 4096;  // event pairs: enough for a 64-field batch (about 12 launches per field)
std::mutex g_mu;
bool g_on = false;
bool g_made = false;
cudaEvent_t g_ev[kPool][2];
int g_stage[kPool];
int g_used = 0;
double g_ms[kNumStages];
long long g_n[kNumStages];
const char* kNames[kNumStages] = {"init", "stats", "consts", "compress", "codebook", "blockbits", "chunkscan",
                                  "pack", "dec_tables", "dec_scan", "huff_decode", "recon", "train"};
}  // namespace

bool prof_on() { return g_on; }

ProfScope::ProfScope(int stage, cudaStream_t s) : stage_(stage), slot_(-1), s_(s) {
  if (!g_on) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_used >= kPool) return;
  slot_ = g_used++;
  g_stage[slot_] = stage;
  cudaEventRecord(g_ev[slot_][0], s_);
}

ProfScope::~ProfScope() {
  if (slot_ >= 0) cudaEventRecord(g_ev[slot_][1], s_);
}

void prof_collect() {
  if (!g_on) return;
  std::lock_guard<std::mutex> lk(g_mu);
  for (int i = 0; i < g_used; ++i) {
    float ms = 0.0f;
    if (cudaEventSynchronize(g_ev[i][1]) == cudaSuccess && cudaEventElapsedTime(&ms, g_ev[i][0], g_ev[i][1]) == cudaSuccess) {
      g_ms[g_stage[i]] += ms;
      g_n[g_stage[i]] += 1;
    }
  }
  g_used = 0;
}

}  // namespace pc

extern "C" {

int pc_profile_enable(int on) {
  using namespace pc;
  std::lock_guard<std::mutex> lk(g_mu);
  if (on && !g_made) {
    for (int i = 0; i < kPool; ++i)
      for (int k = 0; k < 2; ++k)
        if (cudaEventCreate(&g_ev[i][k]) != cudaSuccess) return PC_ERR_CUDA;
    g_made = true;
  }
  g_on = on != 0;
  g_used = 0;
  return PC_OK;
}

int pc_profile_read(double* ms, long long* launches, int n) {
  using namespace pc;
  std::lock_guard<std::mutex> lk(g_mu);
  for (int i = 0; i < kNumStages && i < n; ++i) {
    if (ms) ms[i] = g_ms[i];
    if (launches) launches[i] = g_n[i];
    g_ms[i] = 0.0;
    g_n[i] = 0;
  }
  return kNumStages;
}

const char* pc_profile_stage_name(int i) {
  using namespace pc;
  return (i >= 0 && i < kNumStages) ? kNames[i] : "";
}

}  // extern "C"
