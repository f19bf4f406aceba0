; Sec. 4.1, Example 4: cutPayoff applied to e of Example 3.  The paper prints
;   (100.0 * disc(t0) * if(t0 < now, 0, payoff(you,me)) +
;   if (model(AAPL,t0+t1) > 100.0,
;       (model(AAPL,t0+t1) - 100.0) * disc(t0+t1) *
;        if(t1+t0 < now, 0, payoff(you,me)), 0.0)
; which separates the discount factor from payoff; in the IL of Sec. 3 the
; discount is part of payoff(t, p1, p2), so each payoff(t, ..) is wrapped as
; if(t < now, 0, payoff(t, ..)) by the definition of cutPayoff.
; Times written without their 0 terms; $0 = t0, $1 = t1, you = 0, me = 1.
(add (mult 100.0 (if (lt (texpr $0) (now)) 0.0 (payoff $0 0 1)))
     (if (lt 100.0 (model 0 (tplus $0 $1)))
         (mult (sub (model 0 (tplus $0 $1)) 100.0)
               (if (lt (texpr (tplus $1 $0)) (now)) 0.0 (payoff (tplus $0 $1) 0 1)))
         0.0))
