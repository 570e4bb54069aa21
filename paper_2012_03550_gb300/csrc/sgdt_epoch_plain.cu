// The update kernels specialised for the default options (no momentum, no
// probe minibatch, the 1/M normaliser of Eq. 18): the same source as
// sgdt_epoch.cu compiled with PLAIN = true in a translation unit of its own,
// so that the two sets of kernels build in parallel.  Leaving the other
// options' branches out of the per-minibatch loop shortens the code the SM
// fetches every minibatch.
#define SGDT_EPOCH_PLAIN_TU 1
#include "sgdt_epoch.cu"
