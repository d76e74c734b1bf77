"""CPU oracle for the near-Clifford shot sampler — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import anything from this package. The product (``libnc`` and its
Python binding) never calls it, and this package never imports the product.
The two share no code: only the seeded circuit generators in ``gen/`` (which
hold none of the method's arithmetic) serve both.

Everything here is plain, slow and FP64, written from the paper:

* ``philox``     Philox4x32-10 (Salmon et al., SC'11) and the draw contract.
* ``circuit``    parser for the extended-Stim subset; flattens REPEAT blocks
                 and assigns physical event / site / record indices.
* ``noise``      the cumulative-hazard jump sampler of Sec. 3.2 in its
                 integer survival form.
* ``strata``     stratified importance sampling (Sec. 3.2): Poisson-binomial
                 stratum weights and exactly-K fault sets drawn from the
                 conditional distribution.
* ``dense``      O-B: a dense 2^N state vector of the physical circuit. The
                 plain definition of what the sampler computes, for N <= ~14.
* ``stabilizer`` O-D: CHP tableau reference + physical Pauli-frame
                 propagation (Clifford circuits, any N).
* ``factored``   O-A: the frame-factored method (Def. 2, Lemma 1/App. A,
                 Sec. 2.4/App. B) written step by step.
* ``records``    detector / observable / postselection assembly shared by the
                 three simulators above.

Pins (tests/test_oracle_*.py): Philox known-answer vectors; closed forms
(cos^2(pi/8), sin^2(theta/2), GHZ parity, T^8 = I, the Fig. 4 example);
noise marginals and a brute-force Bernoulli comparison of the sampler;
stratum weights against the binomial closed form and enumeration, the
stratified sampler's path probabilities against the enumerated conditional
distribution;
O-D == O-B and O-A == O-B record-for-record (and P(m=1) to 1e-12) on random
small circuits; O-A == O-D on the d=5 surface-code memory; mirror circuits.

Parity unpinned: O-A's amplitudes at active dimension k > 14 in general (the
dense oracle cannot reach them). What pins them there: invariants, mirror
circuits, and closed-form measurement probabilities along a k = 16 / 18
cascade on a product of entangled two-qubit blocks.
"""
