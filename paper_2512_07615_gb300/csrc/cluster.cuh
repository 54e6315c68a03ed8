// Thread-block cluster support for the rounding kernel: several CTAs (one per
// SM) work on one rounding job.  The leader CTA (rank 0) runs the job; the
// other CTAs of the cluster join it for the FP64 one-sided Jacobi of each
// centre matrix, whose column pairs are spread over all CTAs of the cluster
// (FP64 runs at a small fraction of the FP32 rate per SM, so the Jacobi is
// bounded by the FP64 pipes and scales with the number of SMs).
//
// Synchronisation never waits without a bound.  Each CTA owns two mbarriers
// (expected arrival count = cluster size) used alternately; a cluster barrier
// is: every thread fences its writes at cluster scope, the CTA synchronises,
// thread t < P arrives (release, cluster scope) on CTA t's mbarrier, and every
// thread polls its own CTA's mbarrier (acquire, cluster scope) until the phase
// completes or the wait limit (ns of %globaltimer) runs out.  Alternating the
// two mbarriers keeps an early arrival for barrier b+1 out of the phase that is
// still collecting barrier b.  A CTA whose wait ran out records ST_TIMEOUT,
// stops arriving and waiting, and skips the remaining work of the launch; the
// others then run out too, so every CTA reaches the exit barrier.  The exit
// barrier has its own mbarrier and a fixed generous limit, and only after it
// does any CTA leave (so no CTA touches the shared memory of one that has
// exited).  The one unbounded wait is the launch handshake that every CTA
// executes before any other work, after initialising its mbarriers.
#pragma once

#include "internal.cuh"

namespace tn {

static constexpr int CL_MAX = 16;                 // largest cluster used

// leader -> workers command (written into every worker's shared memory)
struct ClusterCmd {
  int op;                 // 0 = exit, 1 = FP64 Jacobi on the job's W64 / V64 (columns in
                          // global memory), 2 = row-partitioned FP64 SVD of site k
  int ncol, len, maxsw;
  int m, n, k, pad;
  double delta, scl;
};

struct __align__(16) ClusterShared {
  unsigned long long bar[2];   // work barriers (alternating)
  unsigned long long bar_exit; // exit barrier
  unsigned long long xbar[2];  // data exchanges (alternating): one local arrival + the bytes expected
  ClusterCmd cmd;
  int flags[2][CL_MAX];        // per-sweep "rotated" flags of every CTA (double buffered)
  int peer_dead;               // set by a CTA of the cluster that gave up waiting
};

// Per-thread view of the cluster (all fields uniform within a CTA).
struct ClusterCtx {
  ClusterShared* sh;           // this CTA's block (same offset in every CTA)
  int P, rank;
  unsigned nb;                 // work barriers passed so far
  unsigned xe;                 // data exchanges completed so far
  bool dead;                   // a wait ran out
  long long limit_ns;          // wait limit of the work barriers
  int* status;
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned cl_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cl_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned long long gtimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// shared::cluster address of the same variable in CTA `rank`
__device__ __forceinline__ unsigned cl_map(const void* p, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ void cl_arrive_remote(const unsigned long long* bar, unsigned rank) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cl_map(bar, rank))
               : "memory");
}
__device__ __forceinline__ bool cl_try_wait(const unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void cl_store_remote(const int* p, unsigned rank, int v) {
  asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(cl_map(p, rank)), "r"(v) : "memory");
}
__device__ __forceinline__ void cl_store_remote(const double* p, unsigned rank, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(cl_map(p, rank)), "d"(v) : "memory");
}
__device__ __forceinline__ void cl_fence() { asm volatile("fence.acq_rel.cluster;" ::: "memory"); }

// Bounded poll of one mbarrier phase by every thread; true when complete.
__device__ __forceinline__ bool cl_poll(const unsigned long long* bar, unsigned parity, long long limit_ns) {
  if (cl_try_wait(bar, parity)) return true;
  const unsigned long long t0 = gtimer_ns();
  for (;;) {
    if (cl_try_wait(bar, parity)) return true;
    if ((long long)(gtimer_ns() - t0) > limit_ns) return false;
  }
}

// Initialise the barriers and meet every CTA of the cluster once (the launch
// handshake).  All threads of every CTA call this first.
__device__ inline void cl_init(ClusterCtx& c, ClusterShared* sh, int* status, long long limit_ns) {
  c.sh = sh;
  c.P = (int)cl_size();
  c.rank = (int)cl_rank();
  c.nb = 0;
  c.xe = 0;
  c.dead = false;
  c.limit_ns = limit_ns;
  c.status = status;
  if (c.P == 1) return;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&sh->bar[0])), "r"(c.P));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&sh->bar[1])), "r"(c.P));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&sh->bar_exit)), "r"(c.P));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&sh->xbar[0])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&sh->xbar[1])), "r"(1));
    sh->cmd.op = 0;
    sh->peer_dead = 0;
    for (int i = 0; i < 2 * CL_MAX; ++i) (&sh->flags[0][0])[i] = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Uniform check of this CTA's liveness before a batch of stores into other
// CTAs: a CTA that gave up waiting has told every CTA so (peer_dead); after
// that nobody sends it anything more, so that it can leave at the exit
// barrier.  False once this CTA or a peer has given up.
__device__ inline bool cl_alive(ClusterCtx& c) {
  if (c.P == 1) return true;
  if (__syncthreads_or(c.dead || *(volatile int*)&c.sh->peer_dead)) c.dead = true;
  return !c.dead;
}

// Cluster-wide barrier with memory ordering at cluster scope.  Returns false
// (uniformly in the CTA) once this CTA has given up waiting, or learnt that a
// peer has.
__device__ inline bool cl_sync(ClusterCtx& c) {
  if (c.P == 1) {
    __syncthreads();
    return true;
  }
  cl_fence();
  const int j = c.nb & 1;
  const unsigned parity = (c.nb >> 1) & 1;
  ++c.nb;
  if (!cl_alive(c)) return false;
  if (threadIdx.x < (unsigned)c.P) cl_arrive_remote(&c.sh->bar[j], threadIdx.x);
  const bool ok = cl_poll(&c.sh->bar[j], parity, c.limit_ns);
  const int fail = __syncthreads_or(!ok);
  if (fail) {
    c.dead = true;
    if (threadIdx.x == 0) atomicOr(c.status, ST_TIMEOUT);
    // no CTA has left yet (nobody leaves before every CTA reached the exit
    // barrier), so every peer can still be told
    if (threadIdx.x < (unsigned)c.P) cl_store_remote(&c.sh->peer_dead, threadIdx.x, 1);
  }
  return !c.dead;
}

// Exit barrier: every CTA arrives once on every CTA's exit mbarrier and waits
// for the others before leaving (30 s at most: far longer than any stretch a
// live CTA spends between two of its stores into another CTA).
__device__ inline void cl_exit(ClusterCtx& c) {
  if (c.P == 1) return;
  cl_fence();
  __syncthreads();
  if (threadIdx.x < (unsigned)c.P) cl_arrive_remote(&c.sh->bar_exit, threadIdx.x);
  const bool ok = cl_poll(&c.sh->bar_exit, 0, 30000000000LL);
  if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(c.status, ST_TIMEOUT);
}

// ---------------------------------------------------------------- data exchanges
// An exchange sends every CTA the same number of bytes from every CTA of the
// cluster with st.async, each store completing its bytes on the receiver's
// exchange mbarrier; the receiver's one arrival announces the total it
// expects.  The arrival of the data is the synchronisation: a CTA that has all
// bytes of exchange e knows every CTA finished the work before it sent, and
// nobody sends exchange e + 2 into the same buffer before it has this CTA's
// exchange e + 1, which it sends only after reading exchange e.

// Announce the bytes of this exchange (thread 0; before this CTA's own sends).
__device__ inline void cl_xchg_expect(ClusterCtx& c, unsigned bytes) {
  if (c.P > 1 && !c.dead && threadIdx.x == 0)
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&c.sh->xbar[c.xe & 1])),
                 "r"(bytes) : "memory");
}

// One double into CTA `rank`'s copy of *p, counted on its current exchange.
__device__ __forceinline__ void cl_xchg_send(const ClusterCtx& c, const double* p, unsigned rank, double v) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];"
               ::"r"(cl_map(p, rank)), "l"(__double_as_longlong(v)), "r"(cl_map(&c.sh->xbar[c.xe & 1], rank))
               : "memory");
}

// Wait (thread 0 polls, bounded by the wait limit in SM clocks) until all
// bytes of this exchange have arrived; then the CTA meets.  False (uniformly)
// once this CTA has given up.
__device__ inline bool cl_xchg_wait(ClusterCtx& c) {
  if (c.P == 1) {
    __syncthreads();
    return true;
  }
  const unsigned j = c.xe & 1, parity = (c.xe >> 1) & 1;
  ++c.xe;
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    int ok = 1;
    if (!c.dead && !cl_try_wait(&c.sh->xbar[j], parity)) {
      const long long t0 = clock64(), lim = 2 * c.limit_ns;     // ~1 cycle per 0.5 ns
      while (!cl_try_wait(&c.sh->xbar[j], parity))
        if (clock64() - t0 > lim) { ok = 0; break; }
    }
    s_ok = ok;
  }
  __syncthreads();
  if (!c.dead && !s_ok) {
    c.dead = true;
    if (threadIdx.x == 0) atomicOr(c.status, ST_TIMEOUT);
    if (threadIdx.x < (unsigned)c.P) cl_store_remote(&c.sh->peer_dead, threadIdx.x, 1);
  }
  return !c.dead;
}

// Leader: write a command into every worker's shared memory, then meet them.
__device__ inline bool cl_command(ClusterCtx& c, int op, int ncol, int len, int maxsw, int m = 0, int n = 0,
                                  int k = 0, double delta = 0.0, double scl = 0.0) {
  if (c.P == 1) return true;
  if (cl_alive(c) && threadIdx.x >= 1 && threadIdx.x < (unsigned)c.P) {
    const unsigned r = threadIdx.x;
    cl_store_remote(&c.sh->cmd.op, r, op);
    cl_store_remote(&c.sh->cmd.ncol, r, ncol);
    cl_store_remote(&c.sh->cmd.len, r, len);
    cl_store_remote(&c.sh->cmd.maxsw, r, maxsw);
    cl_store_remote(&c.sh->cmd.m, r, m);
    cl_store_remote(&c.sh->cmd.n, r, n);
    cl_store_remote(&c.sh->cmd.k, r, k);
    cl_store_remote(&c.sh->cmd.delta, r, delta);
    cl_store_remote(&c.sh->cmd.scl, r, scl);
  }
  return cl_sync(c);
}

// ---------------------------------------------------------------- FP64 Jacobi over the cluster
// One-sided Jacobi on the ncol rows of W (each of length len, stride ldw) with
// V (ncol x ncol, stride ldv) accumulating the rotations, both in GLOBAL memory
// (read and written at L2, never through L1).  Same pair order (round-robin
// tournament), per-pair arithmetic (half-warp per pair, lanes striding by 16,
// xor-shuffle sums) and stopping test as the single-CTA jacobi_cols_hw<double>,
// so the result does not depend on the cluster size.  Pair p of a round is
// handled by CTA p mod P.  Called by all threads of every CTA of the cluster;
// returns the sweeps used (maxsw if not converged), uniformly.
__device__ inline int jacobi64_cluster(ClusterCtx& c, double* W, int ldw, double* V, int ldv, int ncol,
                                       int len, int maxsw) {
  const int gthreads = c.P * blockDim.x;
  const int gtid = c.rank * blockDim.x + threadIdx.x;
  for (int idx = gtid; idx < ncol * ncol; idx += gthreads)
    __stcg(V + (size_t)(idx / ncol) * ldv + idx % ncol, (idx / ncol == idx % ncol) ? 1.0 : 0.0);
  if (!cl_sync(c) && c.P > 1) return maxsw;
  if (ncol < 2) return 0;
  const int np = (ncol + 1) & ~1;
  const int hl = threadIdx.x & 15, hw = threadIdx.x >> 4, nhw = blockDim.x >> 4;
  const unsigned mask = (threadIdx.x & 16) ? 0xffff0000u : 0x0000ffffu;
  const double tolT = 16.0 * 2.220446049250313e-16 * sqrt((double)len);
  int sweep = 0;
  for (; sweep < maxsw; ++sweep) {
    int rotated = 0;
    for (int rnd = 0; rnd < np - 1; ++rnd) {
      if (!c.dead) {
        for (int p = hw * c.P + c.rank; p < np / 2; p += nhw * c.P) {
          int a, b;
          if (p == 0) { a = rnd; b = np - 1; }
          else { a = (rnd + p) % (np - 1); b = (rnd - p + (np - 1)) % (np - 1); }
          const bool live = a < ncol && b < ncol;
          if (a > b) { int t = a; a = b; b = t; }
          double al = 0.0, be = 0.0, ga = 0.0;
          double* wa = W + (size_t)a * ldw;
          double* wb = W + (size_t)b * ldw;
          if (live)
            for (int i = hl; i < len; i += 16) {
              const double x = __ldcg(wa + i), y = __ldcg(wb + i);
              al += x * x; be += y * y; ga += x * y;
            }
#pragma unroll
          for (int o = 8; o > 0; o >>= 1) {
            al += __shfl_xor_sync(mask, al, o, 16);
            be += __shfl_xor_sync(mask, be, o, 16);
            ga += __shfl_xor_sync(mask, ga, o, 16);
          }
          if (!live || ga == 0.0 || al < 1e-250 || be < 1e-250 || fabs(ga) <= tolT * sqrt(al) * sqrt(be))
            continue;
          const double zeta = (be - al) / (2.0 * ga);
          const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + hypot(1.0, zeta));
          const double cc = 1.0 / sqrt(1.0 + t * t), ss = cc * t;
          for (int i = hl; i < len; i += 16) {
            const double x = __ldcg(wa + i), y = __ldcg(wb + i);
            __stcg(wa + i, cc * x - ss * y);
            __stcg(wb + i, ss * x + cc * y);
          }
          double* va = V + (size_t)a * ldv;
          double* vb = V + (size_t)b * ldv;
          for (int i = hl; i < ncol; i += 16) {
            const double x = __ldcg(va + i), y = __ldcg(vb + i);
            __stcg(va + i, cc * x - ss * y);
            __stcg(vb + i, ss * x + cc * y);
          }
          rotated = 1;
        }
      }
      if (rnd == np - 2) {
        // this CTA's flag for the sweep into every CTA's slot (double buffered by sweep)
        const int any = __syncthreads_or(rotated);
        if (c.P > 1) {
          if (cl_alive(c) && threadIdx.x < (unsigned)c.P) cl_store_remote(&c.sh->flags[sweep & 1][c.rank], threadIdx.x, any);
        } else if (threadIdx.x == 0) {
          c.sh->flags[sweep & 1][0] = any;
        }
      }
      cl_sync(c);
    }
    if (c.dead) return maxsw;
    int any = 0;
    for (int r = 0; r < c.P; ++r) any |= ((volatile int*)c.sh->flags[sweep & 1])[r];
    __syncthreads();
    if (!any) break;
  }
  return sweep;
}

}  // namespace tn
