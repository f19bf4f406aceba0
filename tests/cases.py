"""Parity cases shared by the GPU tests and the CPU emulation tests: market
specs and payoff programs (workloads plus stress programs exercising nested
loopif, lookback, history, now/texpr, nat arithmetic and party folding)."""
import workloads as W

SPECS = {
    "1u_1d": W.MarketSpec([100.0], [0.2], [[1.0]], 0.03, [365]),
    "2u_12d": W.MarketSpec([100.0, 50.0], [0.25, 0.4], W.const_corr(2, -0.3), 0.01,
                           [30 * k for k in range(1, 13)]),
    "3u_5d": W.worst_of_autocall().market,
    "3u_365d": W.daily_barrier().market,
    "4u_irregular": W.MarketSpec([1.0, 2.0, 3.0, 4.0], [0.1, 0.2, 0.3, 0.5],
                                 W.const_corr(4, 0.4), 0.05,
                                 [1, 2, 7, 30, 31, 90, 180, 181, 365, 700, 701, 1000, 3650]),
    "1u_9d": W.MarketSpec([1.0], [0.3], [[1.0]], 0.0, list(range(10, 100, 10))),
}


M2 = W.MarketSpec([100.0, 50.0], [0.25, 0.4], W.const_corr(2, 0.3), 0.02,
                  [30 * k for k in range(1, 13)], now=0,
                  history=[[98.0, 51.0], [97.0, 52.5], [101.0, 49.0]], hist_days=[-1, -2, -3])
M2_LATER = W.MarketSpec([100.0, 50.0], [0.25, 0.4], W.const_corr(2, 0.3), 0.02,
                        [30 * k for k in range(1, 11)], now=2,
                        history=[[99.0, 50.5], [98.0, 51.0]], hist_days=[-30, -60])

M3 = W.MarketSpec([100.0, 50.0, 25.0], [0.2, 0.3, 0.25], W.const_corr(3, 0.4), 0.01,
                  [365 * k for k in range(1, 6)])
M3_MONTHLY = W.MarketSpec([100.0, 100.0, 100.0], [0.2, 0.3, 0.25], W.const_corr(3, 0.6), 0.01,
                          [30 * k for k in range(1, 13)])

STRESS = {
    # double barrier: two compares with different levels -> per-iteration loop step
    "double_barrier": ("(loopif (or (le (model 0 0) 90.0) (lt 56.0 (model 1 0))) 0.0 "
                       "(mult (model 0 0) (payoff 0 0 1)) 11)", [], M2, 100.0),
    # knock-out on a worst-of ratio, literal rebate -> whole-loop instruction
    "worst_knockout": ("(loopif (le (min (div (model 0 0) 100.0) (div (model 1 0) 50.0)) 0.85) 0.25 "
                       "(mult (max (sub (div (model 0 0) 100.0) 1.0) 0.0) (payoff 0 0 1)) $0)", [12], M2, 1.0),
    # worst-of on S_i / S0_i with unequal S0 (fused reduce with divide scales)
    "autocall_scaled": (W.autocall_text([100.0, 50.0, 25.0]), [], M3, 1.0),
    # and-chain of barrier tests and a weighted basket (fused ops, mult scales)
    "basket_and": ("(loopif (and (and (le (model 0 0) 80.0) (le (model 1 0) 80.0)) (le (model 2 0) 80.0)) "
                   "(mult (add (add (mult (model 0 0) 0.5) (mult 0.3 (model 1 0))) (mult (model 2 0) 0.2)) "
                   "(payoff 0 0 1)) (mult (max (sub (add (add (model 0 0) (model 1 0)) (model 2 0)) 300.0) 0.0) "
                   "(payoff 0 0 1)) 12)", [], M3_MONTHLY, 100.0),
    # nested loopif: outer window $0 on label 0, inner window $1 on label 1
    "nested_loops": ("(loopif (lt 105.0 (model 0 0)) "
                     "(loopif (lt (model 1 0) 48.0) (mult (sub (model 0 0) (model 1 0)) (payoff 0 0 1)) "
                     "(mult 2.0 (payoff 0 0 1)) $1) "
                     "(mult (max (sub (model 1 0) 50.0) 0.0) (payoff 0 0 1)) $0)", [6, 3], M2, 50.0),
    # lookback inside a loop: pays S(t0) - S(t0 - 2) on the first date S > 110
    "lookback": ("(loopif (lt 110.0 (model 0 0)) (mult (sub (model 0 0) (model 0 -2)) (payoff 0 0 1)) "
                 "(mult (neg (model 1 -1)) (payoff 0 1 0)) 11)", [], M2, 100.0),
    # history (negative ordinals), texpr / now / nat arithmetic, parties
    "history_now": ("(add (mult (sub (model 0 3) (model 0 -2)) (payoff 3 0 1)) "
                    "(if (lt (texpr (tplus $0 1)) (now)) 0.0 "
                    "(mult (div 1.0 (model 1 $0)) (payoff $0 1 0))))", [4], M2, 100.0),
    "third_party_zero": ("(add (mult (model 0 5) (payoff 5 0 2)) (mult (model 1 5) (payoff 5 0 1)))",
                         [], M2, 50.0),
    "nat_ops": ("(if (and (eq (sub (texpr 3) (nat 5)) (nat 0)) (le (max (texpr $0) (nat 2)) (mult (nat 2) (texpr 2)))) "
                "(mult (min (model 0 1) (model 1 2)) (payoff 2 0 1)) (neg (model 0 1)))", [3], M2, 100.0),
    # the compile example of Sec. 4 after cutPayoff, priced at now = 2 on a
    # market whose history holds the first two dates (Theorem 5 usage)
    "cut_example_now2": ("(add (mult 100.0 (if (lt (texpr $0) (now)) 0.0 (payoff $0 0 1))) "
                         "(if (lt 100.0 (model 0 (tplus $0 $1))) "
                         "(mult (sub (model 0 (tplus $0 $1)) 100.0) "
                         "(if (lt (texpr (tplus $1 $0)) (now)) 0.0 (payoff (tplus $0 $1) 0 1))) 0.0))",
                         [1, 5], M2_LATER, 100.0),
}


def workload_cases():
    c1, c2, c3 = W.european_call(), W.worst_of_autocall(), W.daily_barrier()
    mk1 = c1.market
    return {
        "european": (c1.il_text, c1.tparams, mk1, c1.notional),
        "european_if": (W.european_if_text(100.0), [1], mk1, 100.0),
        "digital": (W.digital_text(100.0), [1], mk1, 1.0),
        "zero_coupon": (W.zero_coupon_text(), [1], mk1, 1.0),
        "forward": (W.forward_text(90.0), [1], mk1, 100.0),
        "exchange": (W.exchange_text(), [12], SPECS["2u_12d"], 100.0),
        "autocall": (c2.il_text, c2.tparams, c2.market, 1.0),
        "daily_barrier": (c3.il_text, c3.tparams, c3.market, 1.0),
        **STRESS,
    }


CASES = workload_cases()


