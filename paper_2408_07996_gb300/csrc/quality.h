// quality.h -- launchers of the event-video quality kernels (Sec. 4.2 metrics).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mcev {

// accumulator slots (unsigned 64-bit words; the distance sums are doubles)
enum {
    QACC_SQ = 0,        // sum over voxels of (a - b)^2
    QACC_NA = 1,        // events in a
    QACC_NB = 2,        // events in b
    QACC_BAD = 3,       // nonzero if a value outside {-1, 0, 1} was seen
    QACC_MATCH_A = 4,   // a events within sqrt(tau2) of a same-polarity b event
    QACC_NONE_A = 5,    // a events whose polarity b lacks entirely
    QACC_SUM_A = 6,     // double: sum of the distances of a's events with d^2 >= QHIST
    QACC_MATCH_B = 7,
    QACC_NONE_B = 8,
    QACC_SUM_B = 9,
    QACC_HIST_A = 16,   // counts of a's events per squared distance 1..QHIST-1 (index = d^2)
    QACC_HIST_B = 16 + 1024,
    QACC_WORDS = 16 + 2048
};

// Squared distances below QHIST are counted per value (the host sums
// count * sqrt(d^2)); only the rare longer ones take a double square root on
// the device, whose FP64 rate is low.
constexpr int QHIST = 1024;

struct QualityArgs {
    const int8_t* a;
    const int8_t* b;
    int32_t W, H, T;
    int32_t tau2;
    int32_t* d2_a;               // optional per-voxel squared distances of a's events (else NULL)
    int32_t* d2_b;
    int32_t* vol0;               // scratch volumes, W*H*T int32 each
    int32_t* vol1;
    unsigned long long* acc;     // QACC_WORDS words
    void* stack;                 // quality_stack_bytes() of scratch for long-line envelopes
};

// Upper bound on the envelope-stack scratch of long column passes (enough
// for every resident thread at lines of up to ~1000; longer lines run fewer
// threads).
constexpr int64_t QUALITY_STACK_BYTES = (int64_t)1 << 31;

// Stack scratch one call on a W x H x T video needs (0 if every column pass
// keeps its stacks in shared memory).
int64_t quality_stack_bytes(int32_t W, int32_t H, int32_t T, int sms);

// Largest extent per axis: keeps every squared lattice distance below 2^30.
constexpr int32_t QUALITY_MAX_EXTENT = 16384;

// Enqueues every kernel on `st`; returns the first launch error.  `launches`
// receives the number of kernels enqueued.
cudaError_t launch_quality(const QualityArgs& A, int sms, cudaStream_t st, int* launches);

}  // namespace mcev
