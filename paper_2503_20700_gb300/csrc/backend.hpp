// Device primitives used by the host planner.
//
// Every floating-point step of the DMRG sweep runs through this interface,
// and the only implementation in the library is the CUDA one (backend_cuda.cu);
// there is no host fallback.  All pointers in task lists are device pointers.
//
// The two workhorses are "segment-sum" primitives with owner-computes
// accumulation (one output block is reduced by one CTA in a fixed order, so
// results are deterministic and need no atomics):
//   place:  C += sum_s alpha_s * op_s(S_s)                  (elementwise)
//   gemm :  C += sum_s alpha_s * op_s(A_s) * op_s(B_s)      (matrix products)
#pragma once
#include <cstddef>
#include <cstdint>
#include <functional>
#include <string>
#include <vector>

namespace dmrg {

// TC_TF32X3: the 3xTF32 split products of SPLIT_TF32 issued on the tcgen05
// tensor cores (H_eff psi only; elsewhere it acts as SPLIT_TF32).
enum class Precision : int { FP64 = 0, SPLIT_TF32 = 1, BF16X9 = 2, TC_TF32X3 = 3 };

struct PlaceSeg {
  const double* src;
  int ld;          // leading dimension of src (row-major)
  int trans;       // 0: src[r*ld + c], 1: src[c*ld + r]
  double alpha;
};
struct PlaceGroup {
  double* dst;
  int rows, cols, ld;
  int seg_begin, seg_count;  // into the segment array
};

struct GemmSeg {
  const double* A;
  const double* B;
  int k;
  int lda, ldb;
  int transA, transB;  // A: 0 -> m x k row-major, 1 -> stored k x m; B: 0 -> k x n, 1 -> stored n x k
  double alpha;
};
struct GemmGroup {
  double* C;
  int m, n, ldc;
  int seg_begin, seg_count;
};

struct EighTask {
  const double* A;  // n x n symmetric, row-major (used as work space: destroyed)
  double* w;        // n eigenvalues, descending
  double* V;        // n x n eigenvectors as rows (row-major storage)
  int n;
};

struct HpsiBlock;
struct HpsiItem;
struct TcItem;
struct SplitJob;
struct HpsiTask;
struct HpsiReduce;
struct TcLaunch;

class Backend {
 public:
  virtual ~Backend() = default;
  virtual std::string name() const = 0;
  virtual void* alloc(size_t bytes) = 0;
  virtual void free(void* p) = 0;
  virtual size_t bytes_in_use() const = 0;
  // device memory the backend can hold in all (bytes), and what the whole
  // device has free now (other contexts included)
  virtual size_t capacity() const { return ~size_t(0); }
  // streaming multiprocessors of the device (the persistent launches' grid)
  virtual int sm_count() const { return 152; }
  // device memory the backend may hold (0: no cap); an allocation beyond it
  // throws "out of device memory"
  virtual void set_budget(size_t bytes) { budget_ = bytes; }
  size_t budget() const { return budget_; }
  // Staging of device buffers to pinned host memory on a side stream.
  //   stage_out(dev, bytes): returns a pinned host copy of dev; the copy runs
  //     on the side stream after all work queued so far on the main stream,
  //     and dev is freed there (stream-ordered) once the copy is done.
  //   stage_in(host, bytes): allocates device memory and copies host into it
  //     on the side stream; returns the device pointer.  The main stream waits
  //     for the copy at the next stage_join() (or at release of the host copy).
  //   stage_join(): the main stream waits for every side-stream copy issued.
  //   host_release(host): frees a pinned copy after its copies completed.
  // called by alloc when an allocation would exceed the budget: frees device
  // memory (e.g. by staging a block out) and returns false when it cannot
  std::function<bool()> make_room;
  virtual void* stage_out(void* dev, size_t bytes) = 0;
  virtual void* stage_in(const void* host, size_t bytes) = 0;
  virtual void stage_join() = 0;
  virtual void host_release(void* host) = 0;
  size_t staged_bytes = 0;       // pinned host bytes currently held
  size_t staged_out_bytes = 0;   // counters of bytes moved (for the accounting)
  size_t staged_in_bytes = 0;
  // bound of every device-side wait of the kernels (nanoseconds; 0: a wait
  // that is not complete at its first probe gives up)
  void set_wait_ns(unsigned long long ns) { wait_ns_ = ns; }
  unsigned long long wait_ns() const { return wait_ns_; }
  virtual size_t device_free() const { return ~size_t(0); }
  virtual void memset0(void* p, size_t bytes) = 0;
  virtual void copy_d2d(void* dst, const void* src, size_t bytes) = 0;
  virtual void copy_h2d(void* dst, const void* src, size_t bytes) = 0;
  virtual void copy_d2h(void* dst, const void* src, size_t bytes) = 0;
  virtual void sync() = 0;
  // Reads and clears the device error flag that bounded waits in kernels set;
  // throws "timeout: ..." when it was set.  Synchronises the stream.
  virtual void check_device_flag() = 0;
  // the stream every primitive is issued on (cudaStream_t)
  virtual void* stream() = 0;

  virtual void place(const std::vector<PlaceGroup>& groups, const std::vector<PlaceSeg>& segs) = 0;
  virtual void gemm(const std::vector<GemmGroup>& groups, const std::vector<GemmSeg>& segs,
                    Precision prec) = 0;

  // Fused H_eff psi (hpsi_fused.cuh); all lists are device arrays prepared by
  // the caller, scratch holds the partial tiles.  flops: algorithmic count
  // of the launch (for the accounting under tag 1).
  virtual void hpsi(const HpsiBlock* blocks, const HpsiItem* items, const HpsiTask* tasks, int ntasks,
                    const HpsiReduce* reds, int nreds, double* scratch, Precision prec,
                    double flops) = 0;
  // The tcgen05 version of the contraction on pre-split operands (hpsi_tc.cuh),
  // and the split of float64 blocks into TF32 hi/lo planes (device job list).
  // tag: profiling counter (1: H_eff psi, 0: other GEMM work)
  virtual void hpsi_tc(const TcLaunch& launch, double flops, int tag = 1) = 0;
  virtual void split(const SplitJob* jobs, int n, float* pool) = 0;

  // Davidson vector algebra on contiguous float64 vectors of length len.
  // out[i] = sum_t V[i*ld + t] * x[t] for i < m   (out is a device array)
  virtual void dots(const double* V, int m, size_t len, size_t ld, const double* x, double* out) = 0;
  // y = beta * y + sum_i c[i] * V[i*ld + :]   (c is a device array of m)
  virtual void combine(double* y, double beta, const double* V, int m, size_t len, size_t ld,
                       const double* c) = 0;
  virtual void axpby(double* y, double a, const double* x, double b, size_t len) = 0;
  // y[t] = x[t] / (d[t] - e) with a guarded denominator (Davidson preconditioner)
  virtual void precondition(double* y, const double* x, const double* d, double e, size_t len) = 0;
  // Symmetric eigendecompositions (FP64, one CTA per matrix).
  virtual void eigh(const std::vector<EighTask>& tasks) = 0;

  // Counters (for the FLOP/byte accounting of the benchmark).
  double gemm_flops = 0.0;   // algorithmic 2*m*n*k summed over segments
  double place_bytes = 0.0;
  // Kernel timing with CUDA events on the launching stream.  While profiling
  // is on, every gemm launch is bracketed by two events and accounted under
  // the current tag (0: other GEMMs, 1: H_eff psi).
  int tag = 0;
  long launches = 0;     // kernel launches issued by this backend
  size_t peak_bytes = 0; // high-water mark of bytes_in_use()
  size_t window_peak = 0;  // high-water mark since the caller last reset it
  // Device-side interval on the backend stream (CUDA events): mark_begin()
  // then mark_end() returns the elapsed milliseconds (synchronising the
  // stream).  Two independent slots (0, 1) so that intervals can nest.
  virtual void mark_begin(int slot = 0) = 0;
  virtual double mark_end(int slot = 0) = 0;
  virtual void set_profile(bool on) = 0;

 protected:
  size_t budget_ = 0;
  unsigned long long wait_ns_ = 2000000000ull;

 public:
  // total device time (ms), algorithmic flops and launches of one tag
  virtual void kernel_stats(int tag, double* ms, double* flops, long* launches) = 0;
};

Backend* make_cuda_backend(int device, std::string* err);

}  // namespace dmrg
