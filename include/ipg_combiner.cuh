/*
 * ipg_combiner.cuh — the hybrid message combiner of Sec. III (Fig. 1) as a CUDA
 * device template, for user-defined combine functions and messages of 4, 8 or
 * 16 bytes.
 *
 * A mailbox is a flag word plus a message slot.  The flag says whether the slot
 * holds a message, which is what lets a vertex tell "no message" apart from a
 * combined message that happens to equal the combine's neutral element (the
 * empty-mailbox problem of compare-and-swap combiners, Sec. III); it also means
 * the combine function needs no neutral element at all.
 *
 *   flag = IPG_MAIL_EMPTY    no message; the slot is meaningless
 *   flag = IPG_MAIL_CLAIMED  one thread holds the first-message lock and is storing
 *   flag = IPG_MAIL_FULL     the slot holds a message
 *
 * Sending message m to a mailbox (ipg_mail_send):
 *   1. flag FULL (acquire load): combine m into the slot with a compare-and-swap
 *      loop — read the slot, combine, CAS; on failure retry with the value the
 *      CAS returned.  If combining leaves the slot unchanged nothing is written.
 *   2. flag EMPTY: try to take the lock (CAS EMPTY -> CLAIMED).  The winner
 *      stores m as the first message and then publishes it by a release store of
 *      FULL, so no thread can see FULL before the message is in place (the
 *      store-then-flag order with a barrier between that Sec. III requires).
 *   3. flag CLAIMED (or the lock was lost): wait until the holder publishes FULL,
 *      then combine as in 1.  The holder only performs one store before it
 *      publishes, so the wait is short; it is still bounded (IPG_MAIL_SPIN_LIMIT
 *      polls), after which the call raises IPG_MAIL_STATUS_TIMEOUT in the
 *      caller's status word and gives up on the message.
 * The CAS loop of 1 is lock-free (a failed CAS means another thread's succeeded)
 * and is bounded too, by IPG_MAIL_CAS_LIMIT retries.
 *
 * The combine function must be commutative and associative, as Pregel
 * combiners are (messages arrive in no fixed order); it is a functor with
 *   __device__ Msg operator()(const Msg& a, const Msg& b) const;
 * Msg must be trivially copyable and 4, 8 or 16 bytes; a 16-byte Msg must be
 * declared alignas(16) (the 128-bit compare-and-swap needs sm_90 or newer).
 * Slots are compared bitwise.
 *
 * Warp pre-combination (ipg_warp_combine): lanes of a warp that send to the
 * same vertex first fold their messages together with __match_any_sync and
 * shuffles, so one lane per distinct destination touches the mailbox.  Hub
 * vertices of power-law graphs receive many messages per warp; this trades a
 * match and a few shuffles for atomics on one hot address.
 *
 * After a complete delivery (every send returned) every flag is EMPTY or FULL,
 * i.e. 0 or 1: the flag array is the has-message array.  To reuse a mailbox,
 * reset its flag to EMPTY once its message has been consumed (a kernel
 * boundary orders the reset before the next superstep's sends).
 *
 * The paper has no GPU counterpart of this file; its combiner is the C11
 * version of Fig. 1 with a lock per vertex.
 */
#pragma once

#include <stdint.h>

#define IPG_MAIL_EMPTY 0u
#define IPG_MAIL_FULL 1u
#define IPG_MAIL_CLAIMED 2u

#define IPG_MAIL_STATUS_TIMEOUT 0x10u /* a wait or a CAS loop ran out (message dropped) */

#ifndef IPG_MAIL_SPIN_LIMIT
#define IPG_MAIL_SPIN_LIMIT (1u << 22)
#endif
#ifndef IPG_MAIL_CAS_LIMIT
#define IPG_MAIL_CAS_LIMIT (1u << 24)
#endif

#ifdef __CUDACC__

#include <string.h>

namespace ipg_mail {

struct alignas(16) Word128 {
    unsigned long long lo, hi;
};

template <int kBytes>
struct WordOf;
template <>
struct WordOf<4> {
    using type = unsigned int;
};
template <>
struct WordOf<8> {
    using type = unsigned long long;
};
template <>
struct WordOf<16> {
    using type = Word128;
};

template <class To, class From>
__device__ __forceinline__ To bits(const From& x) {
    static_assert(sizeof(To) == sizeof(From), "size mismatch");
    To t;
    memcpy(&t, &x, sizeof(To));
    return t;
}

__device__ __forceinline__ bool same(unsigned int a, unsigned int b) { return a == b; }
__device__ __forceinline__ bool same(unsigned long long a, unsigned long long b) { return a == b; }
__device__ __forceinline__ bool same(const Word128& a, const Word128& b) { return a.lo == b.lo && a.hi == b.hi; }

__device__ __forceinline__ unsigned int load_acquire(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void store_release(unsigned int* p, unsigned int v) {
    asm volatile("st.release.gpu.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// single-copy-atomic reads of a 4- or 8-byte slot; a 16-byte read may tear, which
// only costs a failed CAS (the CAS compares all 16 bytes atomically)
__device__ __forceinline__ unsigned int load_relaxed(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.relaxed.gpu.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long load_relaxed(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ Word128 load_relaxed(const Word128* p) {
    Word128 v;
    v.lo = load_relaxed(&p->lo);
    v.hi = load_relaxed(&p->hi);
    return v;
}

__device__ __forceinline__ unsigned int cas(unsigned int* p, unsigned int c, unsigned int v) {
    return atomicCAS(p, c, v);
}
__device__ __forceinline__ unsigned long long cas(unsigned long long* p, unsigned long long c, unsigned long long v) {
    return atomicCAS(p, c, v);
}
__device__ __forceinline__ Word128 cas(Word128* p, Word128 c, Word128 v) { return atomicCAS(p, c, v); }

}  // namespace ipg_mail

// combine m into a slot that already holds a message (step 1); returns false if
// the retry bound ran out (IPG_MAIL_STATUS_TIMEOUT raised)
template <class Combine, class Msg>
__device__ __forceinline__ bool ipg_mail_cas_combine(Msg* slot, const Msg& m, unsigned int* status) {
    static_assert(sizeof(Msg) == 4 || sizeof(Msg) == 8 || sizeof(Msg) == 16, "messages are 4, 8 or 16 bytes");
    using W = typename ipg_mail::WordOf<sizeof(Msg)>::type;
    W* ws = reinterpret_cast<W*>(slot);
    W cur = ipg_mail::load_relaxed(ws);
    const Combine combine{};
    for (unsigned int i = 0; i < IPG_MAIL_CAS_LIMIT; ++i) {
        const W nxt = ipg_mail::bits<W>(combine(ipg_mail::bits<Msg>(cur), m));
        // unchanged: done without a write — for 16 bytes only once a CAS has shown
        // that `cur` was a whole value rather than two halves of different writes
        if (sizeof(Msg) <= 8 && ipg_mail::same(nxt, cur)) return true;
        const W prev = ipg_mail::cas(ws, cur, nxt);
        if (ipg_mail::same(prev, cur)) return true;
        cur = prev;
    }
    atomicOr(status, IPG_MAIL_STATUS_TIMEOUT);
    return false;
}

// Deliver m to the mailbox (flag, slot).  Returns 1 if it was the mailbox's first
// message (the caller can record the receiver exactly once), 0 if it was combined
// into an existing one, -1 if a bounded wait ran out (IPG_MAIL_STATUS_TIMEOUT is
// raised in *status and the message is not delivered).  spin_limit bounds the
// polls of a CLAIMED flag (step 3).
template <class Combine, class Msg>
__device__ __forceinline__ int ipg_mail_send(unsigned int* flag, Msg* slot, const Msg& m, unsigned int* status,
                                             unsigned int spin_limit = IPG_MAIL_SPIN_LIMIT) {
    unsigned int f = ipg_mail::load_acquire(flag);
    if (f == IPG_MAIL_EMPTY) {
        if (atomicCAS(flag, IPG_MAIL_EMPTY, IPG_MAIL_CLAIMED) == IPG_MAIL_EMPTY) {
            *slot = m;
            ipg_mail::store_release(flag, IPG_MAIL_FULL);
            return 1;
        }
        f = IPG_MAIL_CLAIMED;  // lost the lock: re-read with acquire below
    }
    if (f != IPG_MAIL_FULL) {
        unsigned int i = 0;
        do {
            if (++i > spin_limit) {
                atomicOr(status, IPG_MAIL_STATUS_TIMEOUT);
                return -1;
            }
            if (i > 32) __nanosleep(32);
            f = ipg_mail::load_acquire(flag);
        } while (f != IPG_MAIL_FULL);
    }
    return ipg_mail_cas_combine<Combine>(slot, m, status) ? 0 : -1;
}

// Fold the messages of lanes in `active` that send to the same vertex `v`.  Every
// lane in `active` must call this with its own (v, m).  Returns true on the one
// lane per distinct v that should send; on that lane *m is the group's combined
// message.
template <class Combine, class Msg>
__device__ __forceinline__ bool ipg_warp_combine(unsigned int active, unsigned int v, Msg* m) {
    static_assert(sizeof(Msg) % 4 == 0, "messages are whole 32-bit words");
    const unsigned int grp = __match_any_sync(active, v);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(grp) - 1;
    unsigned int rest = grp & ~(1u << leader);
    if (rest) {
        const Combine combine{};
        Msg acc = *m;
        unsigned int words[sizeof(Msg) / 4];
        memcpy(words, m, sizeof(Msg));
        while (rest) {
            const int src = __ffs(rest) - 1;
            rest &= rest - 1;
            unsigned int got[sizeof(Msg) / 4];
#pragma unroll
            for (int q = 0; q < (int)(sizeof(Msg) / 4); ++q) got[q] = __shfl_sync(grp, words[q], src);
            Msg other;
            memcpy(&other, got, sizeof(Msg));
            if (lane == leader) acc = combine(acc, other);
        }
        *m = acc;
    }
    return lane == leader;
}

#endif /* __CUDACC__ */
