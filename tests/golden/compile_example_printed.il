; Sec. 4, Example 3: the payoff expression e as the paper prints it,
;   (100.0 * payoff(t0,you,me)) +
;   if (model(AAPL,t0+t1) > 100.0,
;       (model(AAPL,t0+t1) - 100.0) * payoff(t0+t1,you,me), 0.0)
; with ">" written as lt with swapped operands, loopif(.., 0) shown as if
; (the rewrite of Sec. 6.1) and time sums written without their 0 terms.
; Names: $0 = t0, $1 = t1, you = 0, me = 1, AAPL = label 0.
(add (mult 100.0 (payoff $0 0 1))
     (if (lt 100.0 (model 0 (tplus $0 $1)))
         (mult (sub (model 0 (tplus $0 $1)) 100.0) (payoff (tplus $0 $1) 0 1))
         0.0))
