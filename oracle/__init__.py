"""FP64 CPU oracle for payoff-expression Monte Carlo pricing.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package may import, call,
link or execute this package.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

The oracle is a plain, slow, obviously-correct restatement of the method of
Annenkov & Elsman, "Certified Compilation of Financial Contracts" (PPDP'18):

* ``cl``      -- the contract language CL (Fig. 1), its trace semantics
                 (Sec. 2), instantiation (Def. 1) and horizon bound.
* ``il``      -- the payoff intermediate language (Sec. 3 grammar), its
                 semantics (Fig. 3), the compiler tau_e / tau_c with the smart
                 constructor tplus (Sec. 4) and cutPayoff (Sec. 4.1).
* ``il_text`` -- a printer/parser for the textual S-expression form of IL
                 (an interface format, no arithmetic of the method).
* ``paths``   -- the path generator the paper leaves open (Sec. 6.2 names an
                 MC engine but does not specify it): Philox4x32-10 (Salmon et
                 al., SC'11), 24-bit uniforms, Box-Muller, a breadth-first
                 bisection Brownian bridge, Cholesky correlation and GBM.
* ``mc``      -- the Monte Carlo driver: per-path payoffs and mean/SE.
* ``closed_forms`` -- Black-Scholes call/put, digital, zero-coupon,
                 forward and Margrabe prices (and call delta / vega) used as
                 pins.
* ``pathwise`` -- per-path derivatives of the payoff in S0_l and sigma_l
                 (central differences of the oracle's own FP64 map on common
                 normals).
* ``mlp``     -- the multilayer perceptron of the learned control variate:
                 softplus layers, weighted squared loss, backpropagation,
                 Adam (an extension of the method, not in the paper).
* ``cv``      -- the delta-hedge martingale control variate for the worst-of
                 autocallable template, its states, hedge-ratio tables and
                 network features (an extension of the method).

Every floating-point computation is FP64.  All functions cite the section,
equation or figure of the paper they follow; readings of ambiguous passages
are listed in the repository's design notes.
"""
