"""B300-native hot path of the phylogenetic Hawkes process (arXiv 2103.03348).

Modules (all compute runs in libhawkes.so, hand-written CUDA for sm_103a):
  hawkes      log-likelihood, gradient and Hessian diagonal (Section 2.1, Eqs. 1, 4, 5);
              the HawkesLogLik autograd.Function
  shard       the same evaluation split over shards with one record exchange
  hmc         adaptively preconditioned HMC over (log globals, log-rates[, trend]) (Section 2.3)
  tree        the phylogenetic Brownian prior in O(M) on the tree (Section 2.2, 2.3.1)
  predictive  posterior-predictive simulation over many parameter settings (Section 4)
  surrogate   the learned MLP gradient surrogate
  synth       seeded synthetic workloads
  peaks       ALU microbenchmarks (roofline denominators)
  build       nvcc build of libhawkes.so (in-tree)
"""
