// common.cuh -- types shared by the host side of the C ABI and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace odegpu {

constexpr int kMaxN = 4;   // largest state dimension of a compiled model
constexpr int kMaxP = 16;  // largest parameter count
constexpr int kMaxA = 8;   // largest accessory count
constexpr int kMaxE = 2;   // largest event count
constexpr int kMaxMC = 8;  // solver-wide model constants

enum Scheme { kRK4 = 0, kRKCK45 = 1 };
enum Prec { kFP64 = 0, kFP32RHS = 1 };
enum TdMode { kTdKeep = 0, kTdT0ToT = 1, kTdShift = 2 };
enum SysStatus {
  kStNone = 0,
  kStTEnd = 1,
  kStEventStop = 2,
  kStEquilibrium = 3,
  kStHminNaN = 4,
  kStStepBudget = 5,
  kStTimeout = 6
};

// Solver-wide settings, passed by value in the kernel parameter block (they
// are the same for all threads: the shared per-solver properties of Sec. 6.5
// and Sec. 6.6 of the paper).
struct Props {
  double rtol[kMaxN];
  double atol[kMaxN];
  double hmax, hmin, grow, shrink;
  // error ratios beyond which 0.9 err^(-1/5) is clamped: (0.9/grow)^5 and
  // (0.9/shrink)^5 (filled in by the host)
  double err_grow, err_shrink;
  int evt_dir[kMaxE];
  double evt_tol[kMaxE];
  int evt_stop[kMaxE];
  int max_eq;
  int events_on;
  int td_mode;
  long long max_steps;
  double mc[kMaxMC];
};

// Everything one integration launch needs.  All arrays are device pointers,
// component-major with stride N (value[c * N + i]).
struct KArgs {
  int N;             // systems in this launch
  int ld;            // stride between components of the per-system arrays (>= N)
  double* td;        // [2][N]  (t0, t1)
  double* y;         // [n][N]
  const double* p;   // [P][N]
  double* acc;       // [A][N]
  int* status;       // [N]
  int* ecnt;         // [E][N]
  long long* nacc;   // [N]  accumulated
  long long* nrej;   // [N]  accumulated
  double* records;   // [n_slices - n_skip][A + n + 1][N] or null
  int n_slices;
  int n_skip;
  double h0;
  int* slices_left;          // per-system slices still to run (served pools), or null:
                             // a system runs min(n_slices, slices_left[i]) slices
  unsigned int* queue_head;  // persistent launches: next queue slot to take
  int queue_mode;            // persistent launches: 1 = warp-aggregated pops of
                             // strided 32-system chunks, 2 = one pop per lane
  unsigned int queue_stride; // mode 1: queue chunk c of 32 slots holds systems
                             // 32 * ((c * queue_stride) mod chunks) + 0..31
  int tab_cap;               // RK4 per-sweep launches: entries of the block-shared
                             // forcing table in dynamic shared memory (0 = none)
  int warp_sync;             // 1: the lanes of a warp start every slice together
  int spt;                   // per-sweep launches: systems per thread (<= 1: one);
                             // thread g takes systems g, g + G, g + 2G, ... (G threads)
  int* flags;                // flags[0] != 0: the watchdog stopped a system
  long long time_limit_ns;   // per-thread run-time limit of one launch (0 = none)
  Props pr;
};

// Control block of a resident serving kernel (serve.cuh), one per served
// model, in device memory; word offsets (each on its own 64-byte line).
enum ServeCtlWord {
  kCtlRingHead = 0,    // admission-ring entries taken (device compare-and-swap)
  kCtlRingTail = 16,   // admission-ring entries published (written by the host)
  kCtlStop = 32,       // != 0: yield at the next slice boundary and exit (host)
  kCtlYieldTail = 48,  // yield-list entries reserved (device atomics)
  kCtlFlags = 64,      // watchdog flag
  kCtlWords = 80
};

// Arguments of the resident serving kernel besides its KArgs (whose slot
// arrays are the model's pool; n_slices is the residency quantum).
struct ServeArgs {
  const unsigned int* ring;      // [ring_cap] slot indices to run, in order
  unsigned int ring_cap;
  unsigned int* ctl;             // control block (ServeCtlWord)
  unsigned long long* yl;        // [yl_cap] yielded slots: (lap << 32) | slot
  unsigned int yl_cap;
  unsigned int* done_cnt;        // per request-table entry: systems finished
  unsigned int done_cap;         // entries of done_cnt
  const int* owner;              // [pool capacity] request-table entry of a slot
  long long idle_ns;             // a warp with no work for this long exits
  int lanes_per_warp;            // threads of a warp that take systems (1 .. 32): few
                                 // systems are spread thinly, a warp's FP64 issue
                                 // costing the same whatever its active threads
};

// Per-model kernel table entry: the kernel function for a (scheme,
// precision, persistent) triple, or null when not compiled.
typedef const void* (*KernelLookup)(int scheme, int prec, int persistent);

const void* kernel_duffing(int scheme, int prec, int persistent);
const void* kernel_keller_miksis(int scheme, int prec, int persistent);
const void* kernel_valve(int scheme, int prec, int persistent);
const void* kernel_bounce(int scheme, int prec, int persistent);
const void* kernel_duffing_lyapunov(int scheme, int prec, int persistent);

// Model dimensions (n, P, A, E) of the compiled hooks; false for an unknown
// model.  The kernel of a model for (scheme, precision, launch form), or null.
bool model_dims(int model, int* n, int* P, int* A, int* E);
constexpr int kNumModels = 5;  // model ids 0 .. kNumModels - 1 (enum ode_model)

// Multiplier for the persistent queue's chunk order: coprime with the number
// of 32-system chunks and near its golden-ratio fraction, so that chunks
// popped one after another lie far apart in the system order.
inline unsigned int queue_stride_for(int n_systems) {
  const unsigned int chunks = (unsigned int)((n_systems + 31) / 32);
  if (chunks <= 2) return 1u;
  unsigned int k = (unsigned int)(0.6180339887498949 * chunks);
  if (k < 1) k = 1;
  for (;; k++) {
    unsigned int a = k, b = chunks;
    while (b) { const unsigned int r = a % b; a = b; b = r; }
    if (a == 1) return k;
  }
}
const void* kernel_for(int model, int scheme, int prec, int persistent);

}  // namespace odegpu
